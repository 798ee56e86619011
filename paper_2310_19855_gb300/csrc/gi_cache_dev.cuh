// Device helpers shared by the cell table (gi_cache.cu) and the tile table (gi_tiles.cu):
// descriptor hashing, radiance quantisation, the resolved-value format, the live rule and the
// last-block step of a resolve.
#pragma once

#include <cuda_fp16.h>
#include <math.h>

#include "gi_internal.cuh"

namespace gi {

// In the touch-list form a block of the update takes at most kUpdBlockRecords records (one
// grid-strided chunk per iteration), so its shared-memory list of first touches can never
// overflow and is flushed once, at the end, with one global atomic: warps never wait for one
// another inside the loop.  The bitmap form stages nothing and runs a resident grid.
constexpr int kUpdThreads = 256;
constexpr int kUpdBlockRecords = 2048;
constexpr int kResThreads = 256;
constexpr unsigned kFull = 0xFFFFFFFFu;

// ---------------------------------------------------------------- bulk reductions
// A cell's whole 32-byte accumulator {u64 r, g, b; u32 count; u32 stamp} in one L2 operation:
// the thread writes {r, g, b, count} to a 32-byte shared-memory slot and the bulk-copy unit adds
// it to global memory as four 64-bit lanes (cp.reduce.async.bulk .add.u64; the count lands in the
// low half of the last lane, where it cannot carry into the stamp: a frame adds far fewer than
// 2^32 to a count and every resolve clears it).  Both addresses 32-byte aligned.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_add_accum(void *dst, const unsigned long long *src_smem) {
    // the generic-proxy writes of the slot become visible to the bulk-copy (async) proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(src_smem);
    const unsigned long long ga = (unsigned long long)__cvta_generic_to_global(dst);
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.u64 [%0], [%1], 32;" ::"l"(ga), "r"(sa)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// ---------------------------------------------------------------- L2 eviction priority
// Cache policies for loads and stores whose lines should leave the L2 before (evict_first) or
// after (evict_last) the others.
__device__ __forceinline__ unsigned long long l2_policy_evict_first() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ unsigned long long l2_policy_evict_last() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint4 ld_cg_hint(const uint4 *ptr, unsigned long long pol) {
    uint4 v;
    asm volatile("ld.global.cg.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(ptr), "l"(pol));
    return v;
}
__device__ __forceinline__ void st_hint(uint4 *ptr, uint4 v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(ptr), "r"(v.x), "r"(v.y),
                 "r"(v.z), "r"(v.w), "l"(pol)
                 : "memory");
}

// ---------------------------------------------------------------- hashing
// xxHash32 of a single 4-byte word with a seed (xxHash specification).
__device__ __forceinline__ uint32_t xxh32_word(uint32_t w, uint32_t seed) {
    uint32_t h = seed + 0x165667B1u + 4u;
    h += w * 0xC2B2AE3Du;
    h = __funnelshift_l(h, h, 17) * 0x27D4EB2Fu;
    h ^= h >> 15;
    h *= 0x85EBCA77u;
    h ^= h >> 13;
    h *= 0xC2B2AE3Du;
    h ^= h >> 16;
    return h;
}

// Bucket ("home" slot) from the first hash, 24-bit fingerprint from the second.
__device__ __forceinline__ void cell_of_key(unsigned long long key, uint32_t mask, uint32_t &home,
                                            uint32_t &tag) {
    uint32_t lo = (uint32_t)key, hi = (uint32_t)(key >> 32);
    home = pcg_hash(lo ^ pcg_hash(hi)) & mask;
    uint32_t fp = xxh32_word(lo, xxh32_word(hi, 0u)) >> 8;
    fp = fp ? fp : 1u;
    tag = (fp << 8) | (home & 0xFFu);
}

__device__ __forceinline__ float pick4(const float (&a)[4], int i) {
    return i == 0 ? a[0] : (i == 1 ? a[1] : (i == 2 ? a[2] : a[3]));
}

// Cell descriptor (Sections 2.2.1-2.2.2): LOD from the float32 squared camera
// distance against the Algorithm-6 thresholds, position quantised with
// floor(p * (1/s_l)) wrapped to 19 bits, dominant-axis direction code (ties
// x > y > z, sign bit decides), leak bit ray_len < s_l.  Every float op is an
// explicit round-to-nearest intrinsic so that no contraction changes a bit.
// `flip` = 1 when the direction source is the probe ray (outgoing = -ray).
__device__ __forceinline__ unsigned long long cell_key(const KeyParams &k, float px, float py, float pz, float sx,
                                                       float sy, float sz, float len, uint32_t flip) {
    const int lod = key_lod(k, px, py, pz);
    float inv = pick4(k.inv_side, lod);
    float side = pick4(k.side, lod);
    uint32_t qx = (uint32_t)__float2int_rd(__fmul_rn(px, inv)) & kQMask;
    uint32_t qy = (uint32_t)__float2int_rd(__fmul_rn(py, inv)) & kQMask;
    uint32_t qz = (uint32_t)__float2int_rd(__fmul_rn(pz, inv)) & kQMask;
    unsigned long long leak = (len < side) ? 1ull : 0ull;
    float ax = fabsf(sx), ay = fabsf(sy), az = fabsf(sz);
    int axis = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    float comp = axis == 0 ? sx : (axis == 1 ? sy : sz);
    uint32_t sgn = (__float_as_uint(comp) >> 31) ^ flip;
    unsigned long long code = (unsigned long long)(2 * axis + (int)sgn);
    return ((unsigned long long)lod << 61) | (leak << 60) | (code << 57) | ((unsigned long long)qx << 38) |
           ((unsigned long long)qy << 19) | (unsigned long long)qz;
}

__device__ __forceinline__ bool isfinite3(float a, float b, float c) {
    return isfinite(a) && isfinite(b) && isfinite(c);
}

// Fixed point of one channel: round-half-even(clamp(r, 0, 32768) * 2^24); NaN -> 0.
__device__ __forceinline__ unsigned long long quantize(float r, uint32_t &bad) {
    bad |= (r >= 0.0f && r <= kRadMax) ? 0u : 1u;
    float c = fminf(fmaxf(r, 0.0f), kRadMax);
    return __float2ull_rn(__fmul_rn(c, 16777216.0f));
}

__device__ __forceinline__ float3 load_resolved(const void *r, uint32_t stride, int f16, uint32_t s) {
    r = static_cast<const char *>(r) + (size_t)s * stride;
    if (f16) {
        const ushort4 h = *reinterpret_cast<const ushort4 *>(r);
        return make_float3(__half2float(__ushort_as_half(h.x)), __half2float(__ushort_as_half(h.y)),
                           __half2float(__ushort_as_half(h.z)));
    }
    const float4 v = *reinterpret_cast<const float4 *>(r);
    return make_float3(v.x, v.y, v.z);
}

// The 4th lane marks a cell resolved without history (its first resolve, or its first since an
// eviction): 1 for such a cell, 0 otherwise.  The surrogate reads it to find cold cells.
__device__ __forceinline__ void store_resolved(void *r, uint32_t stride, int f16, uint32_t s, float3 v, bool cold) {
    r = static_cast<char *>(r) + (size_t)s * stride;
    if (f16) {
        ushort4 h;
        h.x = __half_as_ushort(__float2half_rn(v.x));
        h.y = __half_as_ushort(__float2half_rn(v.y));
        h.z = __half_as_ushort(__float2half_rn(v.z));
        h.w = cold ? (unsigned short)0x3C00u : (unsigned short)0u;
        *reinterpret_cast<ushort4 *>(r) = h;
    } else {
        *reinterpret_cast<float4 *>(r) = make_float4(v.x, v.y, v.z, cold ? 1.0f : 0.0f);
    }
}

// a cell answers queries once resolved, until it is evicted
__device__ __forceinline__ bool answers(uint32_t stamp, const LiveRule &r) {
    return stamp != 0u && (!r.has_lr || (r.lr - (stamp - 1u)) < r.evict);
}

// Newly occupied slots added per warp, then the last warp to finish (a ticket over all nwarps
// warps of the launch) resets the touch count and publishes the occupancy, followed by the frame it
// belongs to, to host-mapped memory.  No block barrier: a warp never waits for the others.
__device__ __forceinline__ void resolve_finish(Counters *ctr, uint32_t *occ_out, uint32_t stamp_now, uint32_t nwarps,
                                               uint32_t fresh_new) {
    fresh_new = __reduce_add_sync(kFull, fresh_new);
    if ((threadIdx.x & 31) == 0) {
        if (fresh_new) atomicAdd(&ctr->occupied, fresh_new);
        __threadfence();
        if (atomicAdd(&ctr->ticket, 1u) == nwarps - 1u) {
            // every warp has read the touch count: reset it for the next frame
            ctr->touch_count = 0u;
            ctr->ticket = 0u;
            // occupancy for the host's compaction decision, then the frame it belongs to
            if (occ_out) {
                reinterpret_cast<volatile uint32_t *>(occ_out)[0] = atomicAdd(&ctr->occupied, 0u);
                __threadfence_system();
                reinterpret_cast<volatile uint32_t *>(occ_out)[1] = stamp_now;
            }
        }
    }
}

} // namespace gi
