// World-space radiance cache (Section 2.2): descriptor, bucket hash +
// fingerprint with linear probing, fixed-point accumulation, resolve with an
// exponential moving average and decay-based eviction, lookups.
//
// Table layout (N = 2^log2_slots slots, structure of arrays):
//   tags     u32[N]     fingerprint << 8 | (home mod 256); 0 = empty
//   accum    Accum[N]   {u64 sum r,g,b; u32 count; u32 stamp}, one 32-byte sector
//   resolved float4[N]  (r, g, b, cold), or half4 with GI_RESOLVED_F16
// plus a spare table of the same shape for compaction, a record of the slots touched
// since the last resolve and a counter line.  The first touch of a cell (its count's
// returning add sees 0) either sets the slot's bit in a bitmap (u32[N/32]), which the
// resolve walks and clears in slot order, or is staged per block in shared memory and
// appended to a touch list (u32[N]).  A cache whose accumulators exceed the L2 takes
// the bitmap (slot-ordered resolve traffic), a smaller one the list (cheaper updates).
//
// A cell is the pair (home, fingerprint): probing runs are shorter than 256
// slots, so a tag, which carries home mod 256, can only match within the run
// of its own home.  The set of cells and their sums are therefore independent
// of the order in which warps insert them.
#include <cuda_fp16.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "gi_cache_dev.cuh"

namespace gi {

// ---------------------------------------------------------------- update
// Find or insert the cell (home, tag): linear probing from the home slot, up to max_probe slots.
// The slots are read four at a time (one 16-byte load of an aligned group), so that a run that
// continues past its first slot costs no further round trip until it leaves the group; an empty
// slot is claimed with atomicCAS (a slot, once claimed, never changes during an update: a failed
// claim moves on to the next slot).  k = slots examined before the answer.  Returns GI_SLOT_NONE
// when the run is longer than max_probe.  (1080p, no warp merge: 63 us against 69 us with one
// 4-byte load per slot.)
__device__ __forceinline__ uint32_t probe_cell(const UpdateArgs &a, uint32_t home, uint32_t tag, uint32_t &k) {
    uint32_t s = home;
    k = 0;
    while (k < a.max_probe) {
        const uint32_t g = s & ~3u, st = s & 3u;
        const uint4 q = __ldcg(reinterpret_cast<const uint4 *>(a.tags + g));
        const uint32_t mt = (q.x == tag ? 1u : 0u) | (q.y == tag ? 2u : 0u) | (q.z == tag ? 4u : 0u) |
                            (q.w == tag ? 8u : 0u);
        const uint32_t me = (q.x == kEmpty ? 1u : 0u) | (q.y == kEmpty ? 2u : 0u) | (q.z == kEmpty ? 4u : 0u) |
                            (q.w == kEmpty ? 8u : 0u);
        const uint32_t m = (mt | me) & (0xFu << st) & 0xFu;
        if (!m) {
            k += 4u - st;
            s = (g + 4u) & a.mask;
            continue;
        }
        const uint32_t j = (uint32_t)(__ffs(m) - 1);
        k += j - st;
        if (k >= a.max_probe) break;
        if ((mt >> j) & 1u) return g + j;
        const uint32_t old = atomicCAS(a.tags + g + j, kEmpty, tag);
        if (old == kEmpty || old == tag) return g + j;
        ++k;
        s = (g + j + 1u) & a.mask;
    }
    k = a.max_probe;
    return GI_SLOT_NONE;
}

// Touch list (a.bitmap NULL): three 64-bit reductions of the sums and a returning add of the
// count, whose old value 0 marks the first touch of the cell this frame; first touches go to the
// block's shared-memory list and then, once per block, to the touch list.
// Bitmap: the group's sums and count in one 32-byte bulk reduction from the thread's 32-byte
// shared-memory slot (rewritten only once its previous reduction has read it), and the slot's bit
// set by a non-returning atomicOr.  The block's shared buffer is the first-touch list in the one
// form and the reduction slots in the other.  The bulk reductions dominate the update's issue: at
// 1080p it ran 60 us, 39 us without any accumulation and 44 us when only every fourth lane issued
// its reduction (sums then wrong: bounds taken to size the cost).  A tensor-map reduction of four
// rows per instruction (cp.reduce.async.bulk.tensor .tile::scatter4 .add.u64) compiles but wrote
// the rows instead of adding them (every cell counted one sample), so it is not used.
// MERGE: hits of a warp that name the same cell are merged first (__match_any_sync on the cell,
// pointer-jumping sums), so one leader per cell probes and accumulates.  Without it every hit is
// its own group: same-cell hits of a warp then reach the same accumulator in separate reductions,
// whose integer sums are the same.  Probe rays of one warp belong to one probe and point in
// different directions, so few of them share a cell: at 1080p the merge cost 9 us of the update
// for ~5 % fewer reductions (update 72 us with it, 63 us without), and on the Cornell box at
// 1080p 41 us against 38 us.  It stays available (GI_MERGE_WARP) for workloads whose warps do hit
// the same cells.
static_assert(kUpdBlockRecords * 4 == kUpdThreads * 32, "one 32-byte reduction slot per thread");
template <int KEY_DIR, bool MERGE>
__device__ __forceinline__ void update_body(const UpdateArgs &a, uint32_t blk, uint32_t nblk) {
    __shared__ __align__(32) unsigned long long s_buf[kUpdBlockRecords / 2];
    uint32_t *s_touch = reinterpret_cast<uint32_t *>(s_buf);
    unsigned long long *s_red = s_buf + 4 * threadIdx.x;
    const bool bitmap = a.bitmap != nullptr;
    __shared__ uint32_t s_n, s_base, s_clamped, s_maxp;
    if (threadIdx.x == 0) {
        s_n = 0;
        s_clamped = 0;
        s_maxp = 0;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)nblk * kUpdThreads;
    uint32_t my_clamped = 0, my_maxp = 0;
    // far hits go to the surrogate while it is trusted (the decision of the whole launch)
    uint32_t route_lod = 4u;
    if (a.route_stats) {
        const float den = __ldg(a.route_stats + 2), err = __ldg(a.route_stats + 1);
        if (den > 0.0f && err <= a.route_trust * den) route_lod = a.route_lod;
    }
    for (unsigned long long base = (unsigned long long)blk * kUpdThreads; base < a.n; base += stride) {
        const unsigned long long i = base + threadIdx.x;
        const bool inr = i < a.n;
        // every plane of an in-range record in one round trip (a miss reads sectors its warp's hits
        // read anyway)
        float len = -1.0f, px = 0.f, py = 0.f, pz = 0.f, sx = 0.f, sy = 0.f, sz = 0.f, r0 = 0.f, r1 = 0.f, r2 = 0.f;
        if (inr) {
            len = __ldcs(a.len + i);
            px = __ldcs(a.p[0] + i);
            py = __ldcs(a.p[1] + i);
            pz = __ldcs(a.p[2] + i);
            const float *const *sd = KEY_DIR == GI_KEY_DIR_NORMAL ? a.nrm : a.dir;
            sx = __ldcs(sd[0] + i);
            sy = __ldcs(sd[1] + i);
            sz = __ldcs(sd[2] + i);
            r0 = __ldcs(a.rad[0] + i);
            r1 = __ldcs(a.rad[1] + i);
            r2 = __ldcs(a.rad[2] + i);
        }
        bool hit = inr && isfinite(len) && len >= 0.0f && isfinite3(px, py, pz);
        const bool miss = inr && len == INFINITY;
        bool far = false;
        unsigned long long q0 = 0, q1 = 0, q2 = 0;
        uint32_t home = 0, tag = 0;
        if (hit) {
            uint32_t bad = 0;
            q0 = quantize(r0, bad);
            q1 = quantize(r1, bad);
            q2 = quantize(r2, bad);
            my_clamped += bad;
            unsigned long long key =
                cell_key(a.kp, px, py, pz, sx, sy, sz, len, KEY_DIR == GI_KEY_DIR_NORMAL ? 0u : 1u);
            cell_of_key(key, a.mask, home, tag);
            // the LOD sits in the descriptor's top bits
            far = (uint32_t)(key >> 61) >= route_lod;
            hit = !far;
        }
        uint32_t cnt = hit ? 1u : 0u;
        unsigned peers = 1u << lane;
        if (MERGE) {
            // one leader per cell adds the group's integer sums (order-independent, so still bit-exact)
            const unsigned hm = __ballot_sync(kFull, hit);
            if (hit) peers = __match_any_sync(hm, ((unsigned long long)home << 32) | tag);
            const unsigned above = peers & (0xFFFFFFFEu << lane);
            int nxt = above ? (__ffs(above) - 1) : -1;
            // pointer-jumping suffix sums along each group's lane list
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
        }
        const bool leader = hit && (peers & ((1u << lane) - 1u)) == 0u;
        uint32_t slot = GI_SLOT_NONE;
        if (leader) {
            uint32_t k;
            slot = probe_cell(a, home, tag, k);
            my_maxp = max(my_maxp, k + 1u);
            if (slot == GI_SLOT_NONE) {
                atomicAdd(&a.ctr->dropped, (unsigned long long)cnt);
            } else {
                Accum *ac = a.accum + (size_t)slot * a.acc_stride;
                if (bitmap) {
                    bulk_wait_read();  // the previous reduction has read the slot
                    s_red[0] = q0;
                    s_red[1] = q1;
                    s_red[2] = q2;
                    s_red[3] = cnt;
                    bulk_add_accum(ac, s_red);
                    const uint32_t bit = 1u << (slot & 31u);
                    atomicOr(a.bitmap + (slot >> 5), bit);
                } else {
                    atomicAdd(&ac->sum[0], q0);
                    atomicAdd(&ac->sum[1], q1);
                    atomicAdd(&ac->sum[2], q2);
                    // the count was cleared by the last resolve: the first adder this frame records the slot
                    if (atomicAdd(&ac->count, cnt) == 0u) s_touch[atomicAdd(&s_n, 1u)] = slot;
                }
            }
        }
        uint32_t my_slot = slot;
        if (MERGE) my_slot = __shfl_sync(kFull, slot, hit ? (__ffs(peers) - 1) : lane);
        if (inr) __stcs(a.slot_ids + i, hit ? my_slot : (far ? GI_SLOT_FAR : (miss ? GI_SLOT_MISS : GI_SLOT_NONE)));
    }
    // the bulk reductions complete (their sums visible) before the block ends
    if (bitmap) bulk_wait_all();
    // block totals of the statistics, one global atomic each
    my_clamped = __reduce_add_sync(kFull, my_clamped);
    my_maxp = __reduce_max_sync(kFull, my_maxp);
    if (lane == 0) {
        if (my_clamped) atomicAdd(&s_clamped, my_clamped);
        atomicMax(&s_maxp, my_maxp);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!bitmap) s_base = s_n ? atomicAdd(&a.ctr->touch_count, s_n) : 0u;
        if (s_clamped) atomicAdd(&a.ctr->clamped, (unsigned long long)s_clamped);
        if (s_maxp) atomicMax(&a.ctr->max_probe, s_maxp);
    }
    if (!bitmap) {
        __syncthreads();
        for (uint32_t j = threadIdx.x; j < s_n; j += kUpdThreads) a.touch[s_base + j] = s_touch[j];
    }
}

template <int KEY_DIR, bool MERGE>
__global__ void __launch_bounds__(kUpdThreads, 8) k_update(UpdateArgs a) {
    update_body<KEY_DIR, MERGE>(a, blockIdx.x, gridDim.x);
}

// the four instantiations of k_update on one stream
static inline void launch_update(const UpdateArgs &a, uint32_t key_dir, bool merge, int blocks, cudaStream_t st) {
    if (key_dir == GI_KEY_DIR_NORMAL) {
        if (merge) k_update<GI_KEY_DIR_NORMAL, true><<<blocks, kUpdThreads, 0, st>>>(a);
        else k_update<GI_KEY_DIR_NORMAL, false><<<blocks, kUpdThreads, 0, st>>>(a);
    } else {
        if (merge) k_update<GI_KEY_DIR_RAY, true><<<blocks, kUpdThreads, 0, st>>>(a);
        else k_update<GI_KEY_DIR_RAY, false><<<blocks, kUpdThreads, 0, st>>>(a);
    }
}

// Grid of k_update: enough blocks that none takes more than kUpdBlockRecords records.
static inline int update_blocks(unsigned long long n) {
    return (int)((n + kUpdBlockRecords - 1) / kUpdBlockRecords);
}

// ---------------------------------------------------------------- resolve


// Touch-list form: 2 list entries per thread and iteration, 4 resident blocks per SM; bitmap
// form: warps that compact the set bits of kResBmWords words into a shared list, then resolve 2
// entries per lane and iteration, 4 blocks per SM.  (1080p: the bitmap form 34 us, against 44 us
// when a thread walked its own word's bits 4 at a time with 3 blocks per SM: a word holds 0 to 32
// touched slots, so those threads' chains were as uneven as their words.)
constexpr int kResListUnroll = 2, kResListBlocksPerSm = 4;
constexpr int kResBmUnroll = 2, kResBmBlocksPerSm = 4, kResBmWords = 16;
// a table has at least 2^10 slots: its bitmap words are a whole number of chunks
static_assert(((1u << 10) / 32u) % kResBmWords == 0, "bitmap chunk must divide the smallest table");

// Resolve up to U touched slots (0xFFFFFFFF = none), their loads issued together: the
// accumulator and, speculatively, the resolved history (a cell without history ignores it):
// mean = sum / (count 2^24); a cell without history (never resolved, or evicted by an earlier
// resolve) takes the mean, the others blend; accumulator cleared, stamp = frame + 1.
template <int U>
__device__ __forceinline__ void resolve_slots(const ResolveArgs &a, const uint32_t (&s)[U], uint32_t &fresh_new) {
    uint4 lo[U], hi[U];
    float3 old[U];
    // accumulators leave the L2 first, resolved values last: the probe pass reads them next
    const unsigned long long pfirst = l2_policy_evict_first(), plast = l2_policy_evict_last();
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (s[u] != 0xFFFFFFFFu) {
            const uint4 *src = reinterpret_cast<const uint4 *>(a.accum + (size_t)s[u] * a.acc_stride);
            lo[u] = ld_cg_hint(src, pfirst);
            hi[u] = ld_cg_hint(src + 1, pfirst);
            old[u] = load_resolved(a.resolved, a.res_stride, a.f16, s[u]);
        }
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
        if (s[u] == 0xFFFFFFFFu) continue;
        const uint32_t stamp = hi[u].w;
        // no history: never resolved, or evicted by an earlier resolve (untouched E frames)
        const bool fresh = stamp == 0u || (a.has_lr && (a.lr - (stamp - 1u)) >= a.evict);
        const unsigned long long s0 = ((unsigned long long)lo[u].y << 32) | lo[u].x;
        const unsigned long long s1 = ((unsigned long long)lo[u].w << 32) | lo[u].z;
        const unsigned long long s2 = ((unsigned long long)hi[u].y << 32) | hi[u].x;
        // mean = sum / (count 2^24): one reciprocal, three products (within an ulp of the quotient)
        const float rc = __frcp_rn((float)hi[u].z) * 5.9604644775390625e-8f;
        const float3 m = make_float3(__ull2float_rn(s0) * rc, __ull2float_rn(s1) * rc, __ull2float_rn(s2) * rc);
        fresh_new += stamp == 0u ? 1u : 0u;
        float3 v = m;
        if (!fresh) {
            const float3 o = old[u];
            v = make_float3(o.x + a.alpha * (m.x - o.x), o.y + a.alpha * (m.y - o.y), o.z + a.alpha * (m.z - o.z));
        }
        if (!a.f16) {
            st_hint(reinterpret_cast<uint4 *>(static_cast<char *>(a.resolved) + (size_t)s[u] * a.res_stride),
                    make_uint4(__float_as_uint(v.x), __float_as_uint(v.y), __float_as_uint(v.z),
                               __float_as_uint(fresh ? 1.0f : 0.0f)),
                    plast);
        } else {
            store_resolved(a.resolved, a.res_stride, a.f16, s[u], v, fresh);
        }
        // the cleared accumulator is next read by the next frame's update
        uint4 *dst = reinterpret_cast<uint4 *>(a.accum + (size_t)s[u] * a.acc_stride);
        st_hint(dst, make_uint4(0u, 0u, 0u, 0u), pfirst);
        st_hint(dst + 1, make_uint4(0u, 0u, 0u, a.stamp_now), pfirst);
    }
}

// touch-list form: U list entries per thread and iteration
template <int U>
__device__ __forceinline__ void resolve_list_body(const ResolveArgs &a, uint32_t blk, uint32_t nblk) {
    const uint32_t n = __ldcg(&a.ctr->touch_count);
    const uint32_t stride = nblk * kResThreads;
    uint32_t fresh_new = 0;
    for (uint32_t i0 = blk * kResThreads + threadIdx.x; i0 < n; i0 += U * stride) {
        uint32_t s[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t i = i0 + u * stride;
            s[u] = i < n ? __ldcs(a.touch + i) : 0xFFFFFFFFu;
        }
        resolve_slots<U>(a, s, fresh_new);
    }
    resolve_finish(a.ctr, a.occ_out, a.stamp_now, nblk * (kResThreads / 32), fresh_new);
}

// bitmap form: a warp takes kResBmWords words (16 x 32 consecutive slots), clears them, writes the
// slots of their set bits in slot order to its shared list (a prefix sum of the words' bit counts
// over the lanes gives each lane its place) and resolves the list U entries per lane at a time:
// every lane gets the same share of the warp's touched slots whatever the words hold.
template <int U>
__device__ __forceinline__ void resolve_bm_body(const ResolveArgs &a, uint32_t blk, uint32_t nblk) {
    __shared__ uint32_t s_list[kResThreads / 32][kResBmWords * 32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t nw = nblk * (kResThreads / 32);
    const uint32_t chunks = a.words / kResBmWords;
    uint32_t fresh_new = 0;
    for (uint32_t c = blk * (kResThreads / 32) + warp; c < chunks; c += nw) {
        const uint32_t wi = c * kResBmWords + lane;
        uint32_t bits = lane < kResBmWords ? __ldcg(a.bitmap + wi) : 0u;
        if (bits) a.bitmap[wi] = 0u;
        const int cnt = __popc(bits);
        int incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += t;
        }
        const int total = __shfl_sync(kFull, incl, 31);
        int pos = incl - cnt;
        while (bits) {
            s_list[warp][pos++] = wi * 32u + (uint32_t)(__ffs(bits) - 1);
            bits &= bits - 1u;
        }
        __syncwarp();
        for (int k = lane; k < total; k += 32 * U) {
            uint32_t sl[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int idx = k + 32 * u;
                sl[u] = idx < total ? s_list[warp][idx] : 0xFFFFFFFFu;
            }
            resolve_slots<U>(a, sl, fresh_new);
        }
        __syncwarp();
    }
    resolve_finish(a.ctr, a.occ_out, a.stamp_now, nw, fresh_new);
}

__device__ __forceinline__ void resolve_body(const ResolveArgs &a, uint32_t blk, uint32_t nblk) {
    if (a.bitmap) resolve_bm_body<kResBmUnroll>(a, blk, nblk);
    else resolve_list_body<kResListUnroll>(a, blk, nblk);
}

__global__ void __launch_bounds__(kResThreads, kResListBlocksPerSm) k_resolve(ResolveArgs a) {
    resolve_list_body<kResListUnroll>(a, blockIdx.x, gridDim.x);
}
__global__ void __launch_bounds__(kResThreads, kResBmBlocksPerSm) k_resolve_bitmap(ResolveArgs a) {
    resolve_bm_body<kResBmUnroll>(a, blockIdx.x, gridDim.x);
}

// ---------------------------------------------------------------- queries

__global__ void k_query_slots(const uint32_t *slot_ids, unsigned long long n, const void *resolved, uint32_t res_stride, int f16,
                              uint32_t slots, float e0, float e1, float e2, float4 *out) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t s = __ldcs(slot_ids + i);
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (s < slots) {
            float3 v = load_resolved(resolved, res_stride, f16, s);
            o = make_float4(v.x, v.y, v.z, 1.0f);
        } else if (s == GI_SLOT_MISS) {
            o = make_float4(e0, e1, e2, 1.0f);
        }
        __stcs(out + i, o);
    }
}

template <int KEY_DIR>
__global__ void k_query_points(UpdateArgs a, const void *resolved, uint32_t res_stride, int f16, LiveRule rule,
                               float4 *out) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < a.n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const float len = a.len[i];
        const float px = a.p[0][i], py = a.p[1][i], pz = a.p[2][i];
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (isfinite(len) && len >= 0.0f && isfinite3(px, py, pz)) {
            const float *src0 = KEY_DIR == GI_KEY_DIR_NORMAL ? a.nrm[0] : a.dir[0];
            const float *src1 = KEY_DIR == GI_KEY_DIR_NORMAL ? a.nrm[1] : a.dir[1];
            const float *src2 = KEY_DIR == GI_KEY_DIR_NORMAL ? a.nrm[2] : a.dir[2];
            unsigned long long key = cell_key(a.kp, px, py, pz, src0[i], src1[i], src2[i], len,
                                              KEY_DIR == GI_KEY_DIR_NORMAL ? 0u : 1u);
            uint32_t home, tag;
            cell_of_key(key, a.mask, home, tag);
            uint32_t s = home;
            for (uint32_t k = 0; k < a.max_probe; ++k) {
                const uint32_t t = word_tag(__ldg(a.tags + s));
                if (t == kEmpty) break;
                if (t == tag) {
                    if (answers(__ldg(&a.accum[(size_t)s * a.acc_stride].stamp), rule)) {
                        float3 v = load_resolved(resolved, res_stride, f16, s);
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
// Re-insert every live cell of the current table into the clean spare table
// (home recovered from the slot and the tag's low byte) and clear the current
// table behind it, so that it is clean when it becomes the spare.
__global__ void k_rebuild(SlotWord *old_tags, Accum *old_acc, const void *old_res, SlotWord *new_tags, Accum *new_acc,
                          void *new_res, uint32_t res_bytes, uint32_t mask, uint32_t max_probe, LiveRule rule,
                          Counters *ctr) {
    uint32_t live = 0, dropped = 0;
    const uint32_t N = mask + 1u;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        const uint32_t t = word_tag(old_tags[s]);
        if (t == kEmpty) continue;
        const uint32_t stamp = old_acc[s].stamp;
        if (answers(stamp, rule)) {
            const uint32_t home = (s - ((s - (t & 0xFFu)) & 0xFFu)) & mask;
            uint32_t ns = home, k = 0;
            for (; k < max_probe; ++k) {
                if (atomicCAS(new_tags + ns, kEmpty, t) == kEmpty) break;
                ns = (ns + 1u) & mask;
            }
            if (k < max_probe) {
                new_acc[ns].stamp = stamp;
                if (res_bytes == 8)
                    reinterpret_cast<uint2 *>(new_res)[ns] = reinterpret_cast<const uint2 *>(old_res)[s];
                else
                    reinterpret_cast<uint4 *>(new_res)[ns] = reinterpret_cast<const uint4 *>(old_res)[s];
                ++live;
            } else {
                ++dropped;
            }
        }
        uint4 *dst = reinterpret_cast<uint4 *>(old_acc + s);
        dst[0] = make_uint4(0u, 0u, 0u, 0u);
        dst[1] = make_uint4(0u, 0u, 0u, 0u);
        old_tags[s] = kEmpty;
    }
    live = __reduce_add_sync(kFull, live);
    dropped = __reduce_add_sync(kFull, dropped);
    if ((threadIdx.x & 31) == 0) {
        if (live) atomicAdd(&ctr->occupied, live);
        if (dropped) atomicAdd(&ctr->dropped, (unsigned long long)dropped);
    }
}

// ---------------------------------------------------------------- table scan for stats
__global__ void k_scan_stats(const SlotWord *tags, const Accum *acc, const uint32_t *bitmap, uint32_t N, LiveRule rule,
                             unsigned long long *out /* occupied, live, touched */) {
    unsigned long long occ = 0, live = 0, touched = 0;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < N; s += gridDim.x * blockDim.x) {
        if (bitmap && (s & 31u) == 0u) touched += __popc(bitmap[s >> 5]);
        if (word_tag(tags[s]) == kEmpty) continue;
        ++occ;
        if (acc[s].count > 0u || answers(acc[s].stamp, rule)) ++live;
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


// ---------------------------------------------------------------- batched passes (many views)
// 6 blocks per SM (40 registers): the work-item loop's registers spilled at 8 (16 views: 701
// against 694 frames/s)
template <int KEY_DIR>
__global__ void __launch_bounds__(kUpdThreads, 6) k_update_batched(const UpdateArgs *args, const uint32_t *prefix,
                                                                   uint32_t nviews) {
    __shared__ UpdateArgs sa;
    GI_BATCHED_ITEMS(prefix, nviews, sa, args, (update_body<KEY_DIR, false>(sa, item, items)));
}

__global__ void __launch_bounds__(kResThreads, kResBmBlocksPerSm) k_resolve_batched(const ResolveArgs *args, const uint32_t *prefix,
                                                                    uint32_t nviews) {
    __shared__ ResolveArgs sa;
    GI_BATCHED_ITEMS(prefix, nviews, sa, args, resolve_body(sa, item, items));
}

uint32_t update_blocks_for(unsigned long long n, uint32_t records_per_block) {
    return (uint32_t)((n + records_per_block - 1) / records_per_block);
}

gi_status launch_update_batched(const UpdateArgs *args, const uint32_t *prefix, uint32_t nviews, uint32_t blocks,
                                int key_dir, cudaStream_t st) {
    if (blocks == 0) return GI_OK;
    if (key_dir == GI_KEY_DIR_NORMAL)
        k_update_batched<GI_KEY_DIR_NORMAL>
            <<<resident_grid(k_update_batched<GI_KEY_DIR_NORMAL>, kUpdThreads, blocks), kUpdThreads, 0, st>>>(
                args, prefix, nviews);
    else
        k_update_batched<GI_KEY_DIR_RAY>
            <<<resident_grid(k_update_batched<GI_KEY_DIR_RAY>, kUpdThreads, blocks), kUpdThreads, 0, st>>>(
                args, prefix, nviews);
    return cuda_status(cudaGetLastError(), "k_update_batched launch");
}

gi_status launch_resolve_batched(const ResolveArgs *args, const uint32_t *prefix, uint32_t nviews, uint32_t blocks,
                                 cudaStream_t st) {
    if (blocks == 0) return GI_OK;
    k_resolve_batched<<<resident_grid(k_resolve_batched, kResThreads, blocks), kResThreads, 0, st>>>(args, prefix,
                                                                                                    nviews);
    return cuda_status(cudaGetLastError(), "k_resolve_batched launch");
}

} // namespace gi

// ==================================================================== host side
struct gi_cache_s {
    gi_cache_config cfg;
    int device;
    uint32_t N, mask;
    int sms;
    int upd_blocks, res_blocks;
    gi::SlotWord *tags[2];
    gi::Accum *accum[2];
    void *resolved[2];
    uint32_t res_bytes;  // 16 (float4) or 8 (half4)
    int cur;
    bool tiles;                  // two-level cache: a slot holds a tile of 64 cells
    uint32_t cells;              // addressable cells: N, or 64 N for tiles
    uint32_t *stamp[2];          // tiles: per-cell stamps, state, MIP values (gi_tiles.cu)
    float4 *state[2];
    float4 *mips[2];
    unsigned long long *omask[2];
    unsigned long long *tmask;   // tiles: cells touched since the last resolve
    uint32_t *cidx;              // tiles: accumulator block of each touched tile
    uint32_t *tlist;             // tiles: tile of each accumulator block
    int tres_blocks;
    uint32_t *touch;
    uint32_t *bitmap;            // touched slots since the last resolve, one bit each
    gi::Counters *ctr;
    volatile uint32_t *occ_host; // mapped pinned {occupied, stamp of the resolve that wrote it}
    uint32_t *occ_dev;           // its device address
    unsigned long long *scan;   // device scratch for stats (2 x u64)
    int64_t last_resolved;
    bool touched_since_resolve;
    bool rebuild_checked;
    uint64_t rebuilds, updates, resolves;
    gi_nrc_t route_nrc;          // far hits to this surrogate (gi_cache_route_far), or NULL
    uint32_t route_lod;
};

namespace gi {

CacheView cache_view(gi_cache_t c) {
    CacheView v;
    v.resolved = c->resolved[c->cur];
    v.resolved_stride = c->res_bytes;
    v.resolved_f16 = c->cfg.resolved_format == GI_RESOLVED_F16;
    v.slots = c->cells;
    return v;
}

static TileArrays tile_arrays(const gi_cache_s *c, int k) {
    TileArrays t;
    t.tags = c->tags[k];
    t.accum = c->accum[k];
    t.stamp = c->stamp[k];
    t.state = c->state[k];
    t.resolved = c->resolved[k];
    t.mips = c->mips[k];
    t.omask = c->omask[k];
    return t;
}

static LiveRule live_rule(const gi_cache_s *c) {
    LiveRule r;
    r.has_lr = c->last_resolved >= 0 ? 1u : 0u;
    r.lr = c->last_resolved >= 0 ? (uint32_t)c->last_resolved : 0u;
    r.evict = c->cfg.evict_frames;
    return r;
}

static bool config_ok(const gi_cache_config *c) {
    if (!c) return false;
    if (c->log2_slots < 10 || c->log2_slots > 28) return false;
    if (!(c->cell_size > 0.0f) || !isfinite(c->cell_size)) return false;
    if (c->num_lods < 1 || c->num_lods > 4) return false;
    if (!(c->alpha > 0.0f && c->alpha <= 1.0f)) return false;
    if (c->evict_frames < 1) return false;
    if (c->max_probe < 1 || c->max_probe > 255) return false;
    if (c->key_dir != GI_KEY_DIR_NORMAL && c->key_dir != GI_KEY_DIR_RAY) return false;
    if (c->resolved_format != GI_RESOLVED_F32 && c->resolved_format != GI_RESOLVED_F16) return false;
    if (!(c->rebuild_load >= 0.25f && c->rebuild_load <= 0.95f)) return false;
    if (c->first_touch > GI_FIRST_TOUCH_BITMAP) return false;
    if (c->tiles > 1) return false;
    if (c->tiles && (c->log2_slots > 22 || c->first_touch != GI_FIRST_TOUCH_AUTO || c->min_samples < 1))
        return false;
    if (c->merge > GI_MERGE_WARP) return false;
    return true;
}

bool hits_ok(const gi_hits *h, uint32_t key_dir) {
    if (!h) return false;
    if (h->n == 0) return true;
    for (int a = 0; a < 3; ++a)
        if (!h->pos[a] || !h->nrm[a] || !h->rad[a]) return false;
    if (!h->ray_len) return false;
    if (key_dir == GI_KEY_DIR_RAY)
        for (int a = 0; a < 3; ++a)
            if (!h->ray_dir[a]) return false;
    return true;
}

UpdateArgs cache_update_args(gi_cache_s *c, const gi_hits *h, const gi_view *v, uint32_t *slot_ids) {
    UpdateArgs a;
    for (int k = 0; k < 3; ++k) {
        a.p[k] = h->pos[k];
        a.nrm[k] = h->nrm[k];
        a.rad[k] = h->rad[k];
        a.dir[k] = h->ray_dir[k];
    }
    a.len = h->ray_len;
    a.slot_ids = slot_ids;
    a.n = h->n;
    a.tags = c->tags[c->cur];
    a.accum = c->accum[c->cur];
    a.acc_stride = 1;
    a.touch = c->touch;
    a.bitmap = c->bitmap;
    a.ctr = c->ctr;
    a.mask = c->mask;
    a.max_probe = c->cfg.max_probe;
    a.kp = key_params(c->cfg.cell_size, c->cfg.num_lods, v);
    a.route_stats = nullptr;
    a.route_trust = 0.0f;
    a.route_lod = 4u;
    if (c->route_nrc && c->route_lod < 4u) {
        bool trained = false;
        nrc_route_inputs(c->route_nrc, &a.route_stats, &a.route_trust, &trained);
        if (!trained) a.route_stats = nullptr;
        a.route_lod = c->route_lod;
    }
    return a;
}

static gi_status maybe_rebuild(gi_cache_s *c, cudaStream_t st) {
    // Only at the first update after a resolve (all accumulators are clear then), from the
    // occupancy that resolve wrote to mapped host memory (skipped while it has not arrived).
    if (c->touched_since_resolve || c->rebuild_checked || c->last_resolved < 0) return GI_OK;
    if (c->occ_host[1] != (uint32_t)c->last_resolved + 1u) return GI_OK;
    c->rebuild_checked = true;
    const double occ = (double)c->occ_host[0];
    if (occ <= (double)c->cfg.rebuild_load * (double)c->N) return GI_OK;
    const int nxt = c->cur ^ 1;
    gi_status s = cuda_status(cudaMemsetAsync(&c->ctr->occupied, 0, sizeof(uint32_t), st), "rebuild memset");
    if (s != GI_OK) return s;
    if (c->tiles) {
        s = tile_rebuild_launch(tile_arrays(c, c->cur), tile_arrays(c, nxt), c->tmask, c->res_bytes, c->mask,
                                c->cfg.max_probe, live_rule(c), c->ctr, c->sms * 8, st);
        if (s != GI_OK) return s;
        c->cur = nxt;
        c->rebuilds++;
        return GI_OK;
    }
    k_rebuild<<<c->sms * 8, 256, 0, st>>>(c->tags[c->cur], c->accum[c->cur], c->resolved[c->cur], c->tags[nxt],
                                           c->accum[nxt], c->resolved[nxt], c->res_bytes, c->mask, c->cfg.max_probe,
                                           live_rule(c), c->ctr);
    s = cuda_status(cudaGetLastError(), "k_rebuild launch");
    if (s != GI_OK) return s;
    c->cur = nxt;
    c->rebuilds++;
    return GI_OK;
}

ResolveArgs cache_resolve_args(gi_cache_s *c, uint32_t frame) {
    ResolveArgs a;
    a.touch = c->touch;
    a.bitmap = c->bitmap;
    a.words = c->N / 32u;
    a.accum = c->accum[c->cur];
    a.acc_stride = 1;
    a.resolved = c->resolved[c->cur];
    a.res_stride = c->res_bytes;
    a.ctr = c->ctr;
    a.alpha = c->cfg.alpha;
    a.stamp_now = frame + 1u;
    a.has_lr = c->last_resolved >= 0;
    a.lr = c->last_resolved >= 0 ? (uint32_t)c->last_resolved : 0u;
    a.evict = c->cfg.evict_frames;
    a.f16 = c->cfg.resolved_format == GI_RESOLVED_F16;
    a.occ_out = c->occ_dev;
    return a;
}

void cache_after_resolve(gi_cache_s *c, uint32_t frame) {
    c->rebuild_checked = false;
    c->last_resolved = frame;
    c->touched_since_resolve = false;
    c->resolves++;
}

gi_status cache_before_update(gi_cache_s *c, cudaStream_t st) {
    gi_status s = maybe_rebuild(c, st);
    if (s == GI_OK) c->updates++;
    return s;
}

void cache_after_update(gi_cache_s *c) { c->touched_since_resolve = true; }
int cache_key_dir(const gi_cache_s *c) { return (int)c->cfg.key_dir; }
bool cache_tiled(const gi_cache_s *c) { return c->tiles; }
int cache_device(const gi_cache_s *c) { return c->device; }
int64_t cache_last_resolved(const gi_cache_s *c) { return c->last_resolved; }
gi_nrc_t cache_route_nrc(const gi_cache_s *c) { return c->route_lod < 4u ? c->route_nrc : nullptr; }

static void free_cache(gi_cache_s *c) {
    for (int k = 0; k < 2; ++k) {
        cudaFree(c->tags[k]);
        cudaFree(c->accum[k]);
        cudaFree(c->resolved[k]);
        cudaFree(c->stamp[k]);
        cudaFree(c->state[k]);
        cudaFree(c->mips[k]);
        cudaFree(c->omask[k]);
    }
    cudaFree(c->tmask);
    cudaFree(c->cidx);
    cudaFree(c->tlist);
    cudaFree(c->touch);
    cudaFree(c->bitmap);
    cudaFree(c->ctr);
    cudaFree(c->scan);
    if (c->occ_host) cudaFreeHost((void *)c->occ_host);
    delete c;
}

// Host copies of a tile table (export).
struct TileHost {
    std::vector<SlotWord> tags;
    std::vector<Accum> accum;
    std::vector<uint32_t> stamp;
    std::vector<float4> state;
    std::vector<float4> mips;
};

static gi_status copy_tiles(const gi_cache_s *c, cudaStream_t st, TileHost &h, bool mips) {
    const size_t N = c->N, E = c->cells;
    h.tags.resize(N);
    h.accum.resize(E);
    h.stamp.resize(E);
    h.state.resize(E);
    gi_status s = cuda_status(cudaStreamSynchronize(st), "export sync");
    const int k = c->cur;
    std::vector<Accum> blocks(E);
    std::vector<uint32_t> cidx(N);
    if (s == GI_OK) s = cuda_status(cudaMemcpy(h.tags.data(), c->tags[k], N * sizeof(SlotWord), cudaMemcpyDeviceToHost), "export");
    if (s == GI_OK) s = cuda_status(cudaMemcpy(blocks.data(), c->accum[k], E * sizeof(Accum), cudaMemcpyDeviceToHost), "export");
    if (s == GI_OK) s = cuda_status(cudaMemcpy(cidx.data(), c->cidx, N * sizeof(uint32_t), cudaMemcpyDeviceToHost), "export");
    // accumulators in slot order: a touched tile's block, zeros for the others
    if (s == GI_OK) {
        memset(h.accum.data(), 0, E * sizeof(Accum));
        for (size_t i = 0; i < N; ++i)
            if (cidx[i] < N)
                memcpy(&h.accum[i * kTileCells], &blocks[(size_t)cidx[i] * kTileCells], kTileCells * sizeof(Accum));
    }
    if (s == GI_OK) s = cuda_status(cudaMemcpy(h.stamp.data(), c->stamp[k], E * sizeof(uint32_t), cudaMemcpyDeviceToHost), "export");
    if (s == GI_OK) s = cuda_status(cudaMemcpy(h.state.data(), c->state[k], E * sizeof(float4), cudaMemcpyDeviceToHost), "export");
    if (s == GI_OK && mips) {
        h.mips.resize(N * kTileMips);
        s = cuda_status(cudaMemcpy(h.mips.data(), c->mips[k], N * kTileMips * sizeof(float4), cudaMemcpyDeviceToHost),
                        "export");
    }
    return s;
}

static bool host_answers(uint32_t stamp, const LiveRule &r) {
    return stamp != 0u && (!r.has_lr || (r.lr - (stamp - 1u)) < r.evict);
}

static gi_status export_sorted(std::vector<gi_cell> &cells, gi_cell *out, uint64_t capacity, uint64_t *count,
                               const char *who) {
    std::sort(cells.begin(), cells.end(), [](const gi_cell &x, const gi_cell &y) { return x.identity < y.identity; });
    *count = cells.size();
    if (cells.size() > capacity) {
        if (capacity > 0) {
            set_error("%s: %zu live cells exceed capacity %llu", who, cells.size(), (unsigned long long)capacity);
            return GI_ERR_CAPACITY;
        }
        return GI_OK;
    }
    if (!cells.empty()) memcpy(out, cells.data(), cells.size() * sizeof(gi_cell));
    return GI_OK;
}

} // namespace gi

using namespace gi;

extern "C" {

gi_status gi_cache_create(const gi_cache_config *cfg, gi_cache_t *out) {
    if (!out) {
        set_error("gi_cache_create: out is NULL");
        return GI_ERR_INVALID_ARG;
    }
    *out = nullptr;
    if (!config_ok(cfg)) {
        set_error("gi_cache_create: configuration out of range");
        return GI_ERR_INVALID_ARG;
    }
    gi_cache_s *c = new gi_cache_s();
    memset(c, 0, sizeof *c);
    c->cfg = *cfg;
    c->N = 1u << cfg->log2_slots;
    c->mask = c->N - 1u;
    c->tiles = cfg->tiles != 0;
    c->cells = c->tiles ? c->N * (uint32_t)kTileCells : c->N;
    c->last_resolved = -1;
    c->res_bytes = cfg->resolved_format == GI_RESOLVED_F16 ? 8u : 16u;
    gi_status s = cuda_status(cudaGetDevice(&c->device), "cudaGetDevice");
    if (s == GI_OK) s = cuda_status(cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device), "sm count");
    const size_t N = c->N, E = c->cells;
    for (int k = 0; k < 2 && s == GI_OK; ++k) {
        s = cuda_status(cudaMalloc(&c->tags[k], N * sizeof(SlotWord)), "cudaMalloc tags");
        if (s == GI_OK) s = cuda_status(cudaMalloc(&c->accum[k], E * sizeof(Accum)), "cudaMalloc accum");
        if (s == GI_OK) s = cuda_status(cudaMalloc(&c->resolved[k], E * c->res_bytes), "cudaMalloc resolved");
        if (s == GI_OK) s = cuda_status(cudaMemset(c->tags[k], 0, N * sizeof(SlotWord)), "memset");
        if (s == GI_OK) s = cuda_status(cudaMemset(c->accum[k], 0, E * sizeof(Accum)), "memset");
        if (s == GI_OK) s = cuda_status(cudaMemset(c->resolved[k], 0, E * c->res_bytes), "memset");
        if (s == GI_OK && c->tiles) {
            s = cuda_status(cudaMalloc(&c->stamp[k], E * sizeof(uint32_t)), "cudaMalloc stamps");
            if (s == GI_OK) s = cuda_status(cudaMalloc(&c->state[k], E * sizeof(float4)), "cudaMalloc state");
            if (s == GI_OK) s = cuda_status(cudaMalloc(&c->mips[k], N * kTileMips * sizeof(float4)), "cudaMalloc mips");
            if (s == GI_OK) s = cuda_status(cudaMemset(c->stamp[k], 0, E * sizeof(uint32_t)), "memset");
            if (s == GI_OK) s = cuda_status(cudaMemset(c->state[k], 0, E * sizeof(float4)), "memset");
            if (s == GI_OK) s = cuda_status(cudaMemset(c->mips[k], 0, N * kTileMips * sizeof(float4)), "memset");
            if (s == GI_OK) s = cuda_status(cudaMalloc(&c->omask[k], N * sizeof(unsigned long long)), "cudaMalloc omask");
            if (s == GI_OK) s = cuda_status(cudaMemset(c->omask[k], 0, N * sizeof(unsigned long long)), "memset");
        }
    }
    // First touches: a slot bitmap walked in slot order by the resolve when the accumulators
    // exceed L2 (its ordered accesses then save DRAM traffic), else a touch list (cheaper updates).
    const bool use_bitmap = !c->tiles && cfg->first_touch != GI_FIRST_TOUCH_LIST;
    if (s == GI_OK && c->tiles) {
        s = cuda_status(cudaMalloc(&c->tmask, N * sizeof(unsigned long long)), "cudaMalloc tile masks");
        if (s == GI_OK) s = cuda_status(cudaMemset(c->tmask, 0, N * sizeof(unsigned long long)), "memset");
        if (s == GI_OK) s = cuda_status(cudaMalloc(&c->cidx, N * sizeof(uint32_t)), "cudaMalloc tile blocks");
        if (s == GI_OK) s = cuda_status(cudaMemset(c->cidx, 0xFF, N * sizeof(uint32_t)), "memset");
        if (s == GI_OK) s = cuda_status(cudaMalloc(&c->tlist, N * sizeof(uint32_t)), "cudaMalloc tile list");
    }
    if (s == GI_OK && use_bitmap) {
        s = cuda_status(cudaMalloc(&c->bitmap, N / 8), "cudaMalloc bitmap");
        if (s == GI_OK) s = cuda_status(cudaMemset(c->bitmap, 0, N / 8), "memset");
    } else if (s == GI_OK && !c->tiles) {
        s = cuda_status(cudaMalloc(&c->touch, N * 4), "cudaMalloc touch");
    }
    if (s == GI_OK) s = cuda_status(cudaMalloc(&c->ctr, sizeof(Counters)), "cudaMalloc counters");
    if (s == GI_OK) s = cuda_status(cudaMemset(c->ctr, 0, sizeof(Counters)), "memset");
    if (s == GI_OK) s = cuda_status(cudaMalloc(&c->scan, 3 * sizeof(unsigned long long)), "cudaMalloc scan");
    if (s == GI_OK) {
        void *hp = nullptr;
        s = cuda_status(cudaHostAlloc(&hp, 2 * sizeof(uint32_t), cudaHostAllocMapped), "cudaHostAlloc");
        if (s == GI_OK) {
            c->occ_host = static_cast<volatile uint32_t *>(hp);
            c->occ_host[0] = 0u;
            c->occ_host[1] = 0u;
            s = cuda_status(cudaHostGetDevicePointer((void **)&c->occ_dev, hp, 0), "cudaHostGetDevicePointer");
        }
    }
    if (s == GI_OK) {
        int per_sm = 0;
        s = cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_update<0, false>, kUpdThreads, 0),
                        "occupancy");
        c->upd_blocks = c->sms * std::max(per_sm, 1);
        c->res_blocks = c->sms * (c->bitmap ? kResBmBlocksPerSm : kResListBlocksPerSm);
        c->tres_blocks = c->sms * tile_resolve_blocks_per_sm();
    }
    if (s == GI_OK) s = cuda_status(cudaDeviceSynchronize(), "create sync");
    if (s != GI_OK) {
        free_cache(c);
        return s;
    }
    *out = c;
    return GI_OK;
}

gi_status gi_cache_destroy(gi_cache_t c) {
    if (!c) return GI_OK;
    cudaError_t e = cudaDeviceSynchronize();
    free_cache(c);
    return cuda_status(e, "gi_cache_destroy");
}

gi_status gi_cache_update(gi_cache_t c, const gi_hits *hits, const gi_view *view, uint32_t *slot_ids,
                          gi_stream_t stream) {
    if (!c) {
        set_error("gi_cache_update: cache is NULL");
        return GI_ERR_INVALID_ARG;
    }
    if (!hits_ok(hits, c->cfg.key_dir)) {
        set_error("gi_cache_update: hits has a NULL plane");
        return GI_ERR_INVALID_ARG;
    }
    if (!view_ok(view)) {
        set_error("gi_cache_update: bad view (size or fov)");
        return GI_ERR_INVALID_ARG;
    }
    if (hits->n > 0 && !slot_ids) {
        set_error("gi_cache_update: slot_ids is NULL");
        return GI_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    gi_status s = maybe_rebuild(c, st);
    if (s != GI_OK) return s;
    c->updates++;
    if (hits->n == 0) return GI_OK;
    UpdateArgs a = cache_update_args(c, hits, view, slot_ids);
    if (c->tiles) {
        TileUpdateArgs ta;
        ta.u = a;
        ta.tmask = c->tmask;
        ta.cidx = c->cidx;
        ta.tlist = c->tlist;
        s = tile_update_launch(ta, (int)c->cfg.key_dir, c->upd_blocks, st);
        if (s == GI_OK) c->touched_since_resolve = true;
        return s;
    }
    // the bitmap form stages nothing per block: a resident grid strides over the records
    const int blocks = c->bitmap ? (int)std::min<unsigned long long>((unsigned long long)c->upd_blocks,
                                                                      (hits->n + kUpdThreads - 1) / kUpdThreads)
                                 : update_blocks(hits->n);
    launch_update(a, c->cfg.key_dir, c->cfg.merge == GI_MERGE_WARP, blocks, st);
    s = cuda_status(cudaGetLastError(), "k_update launch");
    if (s == GI_OK) c->touched_since_resolve = true;
    return s;
}

gi_status gi_cache_route_far(gi_cache_t c, gi_nrc_t nrc, uint32_t far_lod) {
    if (!c || c->tiles) {
        set_error("gi_cache_route_far: NULL cache or a tile cache");
        return GI_ERR_INVALID_ARG;
    }
    c->route_nrc = far_lod < 4u ? nrc : nullptr;
    c->route_lod = far_lod;
    return GI_OK;
}

gi_status gi_cache_resolve(gi_cache_t c, uint32_t frame, gi_stream_t stream) {
    if (!c) {
        set_error("gi_cache_resolve: cache is NULL");
        return GI_ERR_INVALID_ARG;
    }
    if (c->last_resolved >= 0 && (int64_t)frame < c->last_resolved) {
        set_error("gi_cache_resolve: frame %u precedes the last resolved frame %lld", frame,
                  (long long)c->last_resolved);
        return GI_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    gi_status s;
    if (c->tiles) {
        TileResolveArgs ta;
        ta.t = tile_arrays(c, c->cur);
        ta.tiles = c->N;
        ta.tmask = c->tmask;
        ta.cidx = c->cidx;
        ta.tlist = c->tlist;
        ta.ctr = c->ctr;
        ta.res_stride = c->res_bytes;
        ta.f16 = c->cfg.resolved_format == GI_RESOLVED_F16;
        ta.alpha = c->cfg.alpha;
        ta.frame = frame;
        ta.stamp_now = frame + 1u;
        ta.has_lr = c->last_resolved >= 0;
        ta.lr = c->last_resolved >= 0 ? (uint32_t)c->last_resolved : 0u;
        ta.evict = c->cfg.evict_frames;
        ta.min_samples = c->cfg.min_samples;
        ta.occ_out = c->occ_dev;
        s = tile_resolve_launch(ta, c->tres_blocks, st);
    } else {
        const ResolveArgs a = cache_resolve_args(c, frame);
        if (a.bitmap)
            k_resolve_bitmap<<<c->res_blocks, kResThreads, 0, st>>>(a);
        else
            k_resolve<<<c->res_blocks, kResThreads, 0, st>>>(a);
        s = cuda_status(cudaGetLastError(), "k_resolve launch");
    }
    if (s != GI_OK) return s;
    cache_after_resolve(c, frame);
    return GI_OK;
}

gi_status gi_cache_query(gi_cache_t c, const gi_query *q, float *out, gi_stream_t stream) {
    if (!c || !q) {
        set_error("gi_cache_query: NULL cache or query");
        return GI_ERR_INVALID_ARG;
    }
    if (q->n == 0) return GI_OK;
    if (!out) {
        set_error("gi_cache_query: out is NULL");
        return GI_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int f16 = c->cfg.resolved_format == GI_RESOLVED_F16;
    int blocks = (int)std::min<unsigned long long>((unsigned long long)c->sms * 16, (q->n + 255) / 256);
    if (q->slot_ids) {
        k_query_slots<<<blocks, 256, 0, st>>>(q->slot_ids, q->n, c->resolved[c->cur], c->res_bytes, f16, c->cells, q->env[0],
                                              q->env[1], q->env[2], reinterpret_cast<float4 *>(out));
    } else {
        if (!q->points || !hits_ok(q->points, c->cfg.key_dir) || q->points->n < q->n || !view_ok(q->view)) {
            set_error("gi_cache_query: by point needs points with n records and a valid view");
            return GI_ERR_INVALID_ARG;
        }
        UpdateArgs a = cache_update_args(c, q->points, q->view, nullptr);
        a.n = q->n;
        if (c->tiles) {
            TileUpdateArgs ta;
            ta.u = a;
            ta.tmask = c->tmask;
            ta.cidx = c->cidx;
            ta.tlist = c->tlist;
            return tile_query_points_launch(ta, tile_arrays(c, c->cur), c->res_bytes, f16, live_rule(c),
                                            reinterpret_cast<float4 *>(out), blocks, (int)c->cfg.key_dir, st);
        }
        if (c->cfg.key_dir == GI_KEY_DIR_NORMAL)
            k_query_points<GI_KEY_DIR_NORMAL><<<blocks, 256, 0, st>>>(a, c->resolved[c->cur], c->res_bytes, f16, live_rule(c),
                                                                      reinterpret_cast<float4 *>(out));
        else
            k_query_points<GI_KEY_DIR_RAY><<<blocks, 256, 0, st>>>(a, c->resolved[c->cur], c->res_bytes, f16, live_rule(c),
                                                                   reinterpret_cast<float4 *>(out));
    }
    return cuda_status(cudaGetLastError(), "k_query launch");
}

gi_status gi_cache_stats(gi_cache_t c, gi_cache_stats_t *out, gi_stream_t stream) {
    if (!c || !out) {
        set_error("gi_cache_stats: NULL argument");
        return GI_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    gi_status s = cuda_status(cudaMemsetAsync(c->scan, 0, 3 * sizeof(unsigned long long), st), "stats memset");
    if (s != GI_OK) return s;
    if (c->tiles) {
        s = tile_scan_launch(tile_arrays(c, c->cur), c->tmask, c->N, live_rule(c), c->scan, c->sms * 4, st);
    } else {
        k_scan_stats<<<c->sms * 4, 256, 0, st>>>(c->tags[c->cur], c->accum[c->cur], c->bitmap, c->N, live_rule(c),
                                                 c->scan);
        s = cuda_status(cudaGetLastError(), "k_scan_stats launch");
    }
    if (s != GI_OK) return s;
    Counters h;
    unsigned long long sc[3];
    s = cuda_status(cudaMemcpyAsync(&h, c->ctr, sizeof h, cudaMemcpyDeviceToHost, st), "stats copy");
    if (s == GI_OK) s = cuda_status(cudaMemcpyAsync(sc, c->scan, sizeof sc, cudaMemcpyDeviceToHost, st), "stats copy");
    if (s == GI_OK) s = cuda_status(cudaStreamSynchronize(st), "stats sync");
    if (s != GI_OK) return s;
    memset(out, 0, sizeof *out);
    out->slots = c->N;
    out->occupied = sc[0];
    out->live = sc[1];
    out->touched = (c->bitmap || c->tiles) ? sc[2] : h.touch_count;
    out->dropped = h.dropped;
    out->clamped = h.clamped;
    out->rebuilds = c->rebuilds;
    out->updates = c->updates;
    out->resolves = c->resolves;
    out->max_probe_seen = h.max_probe;
    out->error_word = h.error_word;
    out->last_resolved = c->last_resolved;
    if (h.error_word) return GI_ERR_DEVICE_FAULT;
    if (h.dropped) return GI_WARN_DROPPED;
    return GI_OK;
}

gi_status gi_cache_export(gi_cache_t c, gi_cell *out, uint64_t capacity, uint64_t *count, gi_stream_t stream) {
    if (!c || !count || (capacity > 0 && !out)) {
        set_error("gi_cache_export: NULL argument");
        return GI_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (c->tiles) {
        TileHost h;
        gi_status s = copy_tiles(c, st, h, false);
        if (s != GI_OK) return s;
        const LiveRule r = live_rule(c);
        std::vector<gi_cell> cells;
        for (uint32_t i = 0; i < c->N; ++i) {
            const uint32_t t = h.tags[i];
            if (t == kEmpty) continue;
            const uint32_t home = (i - ((i - (t & 0xFFu)) & 0xFFu)) & c->mask;
            const uint64_t tid = ((uint64_t)home << 24) | (uint64_t)(t >> 8);
            for (uint32_t k = 0; k < (uint32_t)kTileCells; ++k) {
                const size_t e = (size_t)i * kTileCells + k;
                const Accum &a = h.accum[e];
                if (!(a.count > 0 || host_answers(h.stamp[e], r))) continue;
                gi_cell cell;
                cell.identity = (tid << 6) | k;
                for (int q = 0; q < 3; ++q) cell.sum[q] = a.sum[q];
                cell.count = a.count;
                cell.stamp = h.stamp[e];
                cell.value[0] = h.state[e].x;
                cell.value[1] = h.state[e].y;
                cell.value[2] = h.state[e].z;
                cell.slot = (uint32_t)e;
                cells.push_back(cell);
            }
        }
        return export_sorted(cells, out, capacity, count, "gi_cache_export");
    }
    const size_t N = c->N;
    const int f16 = c->cfg.resolved_format == GI_RESOLVED_F16;
    std::vector<SlotWord> tags(N);
    std::vector<Accum> acc(N);
    std::vector<unsigned char> res(N * c->res_bytes);
    gi_status s = cuda_status(cudaStreamSynchronize(st), "export sync");
    if (s == GI_OK) s = cuda_status(cudaMemcpy(tags.data(), c->tags[c->cur], N * sizeof(SlotWord), cudaMemcpyDeviceToHost), "export");
    if (s == GI_OK)
        s = cuda_status(cudaMemcpy(acc.data(), c->accum[c->cur], N * sizeof(Accum), cudaMemcpyDeviceToHost), "export");
    if (s == GI_OK)
        s = cuda_status(cudaMemcpy(res.data(), c->resolved[c->cur], res.size(), cudaMemcpyDeviceToHost), "export");
    if (s != GI_OK) return s;
    const LiveRule r = live_rule(c);
    std::vector<gi_cell> cells;
    for (uint32_t i = 0; i < c->N; ++i) {
        const uint32_t t = tags[i];
        if (t == kEmpty) continue;
        const Accum &a = acc[i];
        const bool live = a.count > 0 || (a.stamp != 0 && (!r.has_lr || (r.lr - (a.stamp - 1u)) < r.evict));
        if (!live) continue;
        gi_cell cell;
        const uint32_t home = (i - ((i - (t & 0xFFu)) & 0xFFu)) & c->mask;
        cell.identity = ((uint64_t)home << 24) | (uint64_t)(t >> 8);
        for (int k = 0; k < 3; ++k) cell.sum[k] = a.sum[k];
        cell.count = a.count;
        cell.stamp = a.stamp;
        if (f16) {
            const __half *h = reinterpret_cast<const __half *>(res.data() + (size_t)i * c->res_bytes);
            for (int k = 0; k < 3; ++k) cell.value[k] = __half2float(h[k]);
        } else {
            const float *f = reinterpret_cast<const float *>(res.data() + (size_t)i * c->res_bytes);
            for (int k = 0; k < 3; ++k) cell.value[k] = f[k];
        }
        cell.slot = i;
        cells.push_back(cell);
    }
    return export_sorted(cells, out, capacity, count, "gi_cache_export");
}

gi_status gi_cache_export_tiles(gi_cache_t c, gi_tile *out, uint64_t capacity, uint64_t *count, gi_stream_t stream) {
    if (!c || !count || (capacity > 0 && !out)) {
        set_error("gi_cache_export_tiles: NULL argument");
        return GI_ERR_INVALID_ARG;
    }
    if (!c->tiles) {
        set_error("gi_cache_export_tiles: the cache holds cells, not tiles");
        return GI_ERR_INVALID_ARG;
    }
    TileHost h;
    gi_status s = copy_tiles(c, (cudaStream_t)stream, h, true);
    if (s != GI_OK) return s;
    const LiveRule r = live_rule(c);
    std::vector<gi_tile> tiles;
    for (uint32_t i = 0; i < c->N; ++i) {
        const uint32_t t = h.tags[i];
        if (t == kEmpty) continue;
        gi_tile tile;
        memset(&tile, 0, sizeof tile);
        for (uint32_t k = 0; k < (uint32_t)kTileCells; ++k) {
            const size_t e = (size_t)i * kTileCells + k;
            if (h.accum[e].count > 0) ++tile.live;
            if (!host_answers(h.stamp[e], r)) continue;
            if (h.accum[e].count == 0) ++tile.live;
            tile.value[k][0] = h.state[e].x;
            tile.value[k][1] = h.state[e].y;
            tile.value[k][2] = h.state[e].z;
            memcpy(&tile.samples[k], &h.state[e].w, sizeof(uint32_t));
        }
        if (!tile.live) continue;
        for (uint32_t k = 0; k < (uint32_t)kTileMips; ++k) {
            const float4 &m = h.mips[(size_t)i * kTileMips + k];
            tile.value[kTileCells + k][0] = m.x;
            tile.value[kTileCells + k][1] = m.y;
            tile.value[kTileCells + k][2] = m.z;
            memcpy(&tile.samples[kTileCells + k], &m.w, sizeof(uint32_t));
        }
        const uint32_t home = (i - ((i - (t & 0xFFu)) & 0xFFu)) & c->mask;
        tile.identity = ((uint64_t)home << 24) | (uint64_t)(t >> 8);
        tile.slot = i;
        tiles.push_back(tile);
    }
    std::sort(tiles.begin(), tiles.end(), [](const gi_tile &x, const gi_tile &y) { return x.identity < y.identity; });
    *count = tiles.size();
    if (tiles.size() > capacity) {
        if (capacity > 0) {
            set_error("gi_cache_export_tiles: %zu tiles exceed capacity %llu", tiles.size(),
                      (unsigned long long)capacity);
            return GI_ERR_CAPACITY;
        }
        return GI_OK;
    }
    if (!tiles.empty()) memcpy(out, tiles.data(), tiles.size() * sizeof(gi_tile));
    return GI_OK;
}

} // extern "C"

// ==================================================================== allocation-free cell means
// One-shot variant of the update pass for callers that cannot allocate device memory: the
// hash table, touch list, counters and per-record slot ids live in one file-scope device array
// (zero at module load, cleared again at the start of every call), so nothing here calls
// cudaMalloc / cudaFree.  Every GPU that loads the library holds this array until exit.
namespace gi {

constexpr uint32_t kNoAllocSlots = 1u << GI_NOALLOC_LOG2_SLOTS;
constexpr size_t kNoAllocTagBytes = (size_t)kNoAllocSlots * sizeof(SlotWord);
constexpr size_t kNoAllocAccumBytes = (size_t)kNoAllocSlots * sizeof(Accum);
constexpr size_t kNoAllocTouchBytes = (size_t)kNoAllocSlots * sizeof(uint32_t);
constexpr size_t kNoAllocSlotIdBytes = (size_t)GI_NOALLOC_MAX_RECORDS * sizeof(uint32_t);
constexpr size_t kNoAllocBytes =
    kNoAllocTagBytes + kNoAllocAccumBytes + kNoAllocTouchBytes + kNoAllocSlotIdBytes + sizeof(Counters);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Host-side addresses of g_noalloc_scratch, one per device (the symbol's name is only a host
// stand-in; the device address must come from cudaGetSymbolAddress with that device current).
static std::mutex g_noalloc_mutex;
static void *g_noalloc_ptr[64];
static int g_noalloc_blocks[64];

static gi_status noalloc_setup(int dev, unsigned char **base, int *blocks) {
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (dev < 0 || dev >= 64) {
        set_error("gi_cell_means_noalloc: device ordinal %d out of range", dev);
        return GI_ERR_INVALID_ARG;
    }
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        gi_status s = cuda_status(cudaGetSymbolAddress(&p, g_noalloc_scratch), "cudaGetSymbolAddress");
        if (s != GI_OK) return s;
        int sms = 0, per_sm = 0;
        s = cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "sm count");
        if (s == GI_OK)
            s = cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_update<0, false>, kUpdThreads, 0),
                            "occupancy");
        if (s != GI_OK) return s;
        g_noalloc_blocks[dev] = sms * std::max(per_sm, 1);
        g_noalloc_ptr[dev] = p;
    }
    *base = static_cast<unsigned char *>(g_noalloc_ptr[dev]);
    *blocks = g_noalloc_blocks[dev];
    return GI_OK;
}

__global__ void k_noalloc_clear(uint4 *p, size_t n16) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n16; i += (size_t)gridDim.x * blockDim.x)
        p[i] = make_uint4(0u, 0u, 0u, 0u);
}

// out[i] = (mean of the cell of record i, 1); (env, 1) for a ray that left the scene; (0, 0, 0, -1)
// for a hit whose cell found no free slot within its probing run (dropped); 0 otherwise.  The mean
// is computed with the same float32 operations as the resolve of a cell without history.
__global__ void k_noalloc_means(const uint32_t *slot_ids, unsigned long long n, const Accum *accum, const float *len,
                                const float *px, const float *py, const float *pz, float e0, float e1, float e2,
                                float4 *out) {
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const uint32_t s = slot_ids[i];
        float4 o = make_float4(0.f, 0.f, 0.f, 0.f);
        if (s < kNoAllocSlots) {
            const Accum a = accum[s];
            const float rc = __frcp_rn((float)a.count) * 5.9604644775390625e-8f;
            o = make_float4(__ull2float_rn(a.sum[0]) * rc, __ull2float_rn(a.sum[1]) * rc, __ull2float_rn(a.sum[2]) * rc,
                            1.0f);
        } else if (s == GI_SLOT_MISS) {
            o = make_float4(e0, e1, e2, 1.0f);
        } else {
            // the update writes GI_SLOT_NONE both for a record that is no hit and for a dropped hit:
            // the record's own hit test (the update's) tells them apart
            const float l = len[i];
            if (isfinite(l) && l >= 0.0f && isfinite3(px[i], py[i], pz[i])) o.w = -1.0f;
        }
        out[i] = o;
    }
}

// stats[0] = hits dropped, stats[1] = hits whose radiance was clamped, from the call's counters
__global__ void k_noalloc_stats(const Counters *ctr, unsigned long long *stats) {
    if (threadIdx.x == 0) {
        stats[0] = ctr->dropped;
        stats[1] = ctr->clamped;
    }
}

} // namespace gi

extern "C" gi_status gi_cell_means_noalloc(const gi_hits *hits, const gi_view *view, float cell_size,
                                           uint32_t num_lods, uint32_t key_dir, const float env[3], float *out,
                                           uint64_t *stats_out, gi_stream_t stream) {
    using namespace gi;
    if (!hits_ok(hits, key_dir) || !view_ok(view) || (hits && hits->n > 0 && !out)) {
        set_error("gi_cell_means_noalloc: NULL record plane or output, or bad view");
        return GI_ERR_INVALID_ARG;
    }
    if (!(cell_size > 0.0f) || !isfinite(cell_size) || num_lods < 1 || num_lods > 4 ||
        (key_dir != GI_KEY_DIR_NORMAL && key_dir != GI_KEY_DIR_RAY)) {
        set_error("gi_cell_means_noalloc: cell_size, num_lods or key_dir out of range");
        return GI_ERR_INVALID_ARG;
    }
    if (hits->n > GI_NOALLOC_MAX_RECORDS) {
        set_error("gi_cell_means_noalloc: %llu records exceed the maximum of %u per call",
                  (unsigned long long)hits->n, (unsigned)GI_NOALLOC_MAX_RECORDS);
        return GI_ERR_INVALID_ARG;
    }
    if (stats_out && (reinterpret_cast<uintptr_t>(stats_out) & 7u)) {
        set_error("gi_cell_means_noalloc: stats_out must be 8-byte aligned");
        return GI_ERR_INVALID_ARG;
    }
    if (hits->n == 0) {
        if (stats_out)
            return cuda_status(cudaMemsetAsync(stats_out, 0, 2 * sizeof(uint64_t), (cudaStream_t)stream),
                               "gi_cell_means_noalloc stats");
        return GI_OK;
    }
    int dev = 0;
    gi_status s = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
    unsigned char *base = nullptr;
    int blocks = 0;
    if (s == GI_OK) s = noalloc_setup(dev, &base, &blocks);
    if (s != GI_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    SlotWord *tags = reinterpret_cast<SlotWord *>(base);
    Accum *accum = reinterpret_cast<Accum *>(base + kNoAllocTagBytes);
    uint32_t *touch = reinterpret_cast<uint32_t *>(base + kNoAllocTagBytes + kNoAllocAccumBytes);
    uint32_t *slot_ids = reinterpret_cast<uint32_t *>(base + kNoAllocTagBytes + kNoAllocAccumBytes + kNoAllocTouchBytes);
    Counters *ctr = reinterpret_cast<Counters *>(base + kNoAllocTagBytes + kNoAllocAccumBytes + kNoAllocTouchBytes +
                                                 kNoAllocSlotIdBytes);
    // the table and the counters must start at zero; the touch list and slot ids are overwritten
    k_noalloc_clear<<<blocks, 256, 0, st>>>(reinterpret_cast<uint4 *>(base),
                                            (kNoAllocTagBytes + kNoAllocAccumBytes) / 16);
    s = cuda_status(cudaGetLastError(), "k_noalloc_clear launch");
    if (s != GI_OK) return s;
    k_noalloc_clear<<<1, 32, 0, st>>>(reinterpret_cast<uint4 *>(ctr), sizeof(Counters) / 16);
    s = cuda_status(cudaGetLastError(), "k_noalloc_clear launch");
    if (s != GI_OK) return s;
    UpdateArgs a;
    for (int k = 0; k < 3; ++k) {
        a.p[k] = hits->pos[k];
        a.nrm[k] = hits->nrm[k];
        a.rad[k] = hits->rad[k];
        a.dir[k] = hits->ray_dir[k];
    }
    a.len = hits->ray_len;
    a.slot_ids = slot_ids;
    a.n = hits->n;
    a.tags = tags;
    a.accum = accum;
    a.acc_stride = 1;
    a.touch = touch;
    a.bitmap = nullptr;
    a.ctr = ctr;
    a.mask = kNoAllocSlots - 1u;
    a.max_probe = 255;
    a.kp = key_params(cell_size, num_lods, view);
    a.route_stats = nullptr;
    a.route_trust = 0.0f;
    a.route_lod = 4u;
    const int ub = update_blocks(hits->n);
    launch_update(a, key_dir, false, ub, st);
    s = cuda_status(cudaGetLastError(), "k_update launch");
    if (s != GI_OK) return s;
    const float e0 = env ? env[0] : 0.0f, e1 = env ? env[1] : 0.0f, e2 = env ? env[2] : 0.0f;
    k_noalloc_means<<<ub, 256, 0, st>>>(slot_ids, hits->n, accum, hits->ray_len, hits->pos[0], hits->pos[1],
                                        hits->pos[2], e0, e1, e2, reinterpret_cast<float4 *>(out));
    s = cuda_status(cudaGetLastError(), "k_noalloc_means launch");
    if (s != GI_OK || !stats_out) return s;
    k_noalloc_stats<<<1, 32, 0, st>>>(ctr, reinterpret_cast<unsigned long long *>(stats_out));
    return cuda_status(cudaGetLastError(), "k_noalloc_stats launch");
}
