// Diagnostics, not a step of the path: the L2 floor of the cache update's accumulation.
//
// gi_cache_update ends, per hit record (the default GI_MERGE_NONE form), in L2 operations on the
// cell's 32-byte accumulator.  List form: three 64-bit additions (the fixed-point sums) and one returning
// 32-bit addition (the count, whose old value flags the first touch).  Bitmap form: one 32-byte
// bulk reduction of the sums and count from shared memory and a non-returning set of the slot's
// bit.  k_diag_atomics issues exactly those operations for a frame's slot ids, with nothing else
// (no record stream, key, probe or slot-id store), so its time is the floor of that form on this
// GPU.
#include "gi_cache_dev.cuh"

namespace gi {

template <bool BITMAP>
__global__ void __launch_bounds__(kUpdThreads, 8) k_diag_atomics(const uint32_t *slot_ids, unsigned long long n,
                                                                  uint32_t slots, Accum *acc, uint32_t *bitmap,
                                                                  uint32_t *first_out) {
    __shared__ __align__(32) unsigned long long s_red[kUpdThreads][4];
    __shared__ uint32_t s_first;
    if (threadIdx.x == 0) s_first = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * kUpdThreads;
    uint32_t first = 0;
    for (unsigned long long base = (unsigned long long)blockIdx.x * kUpdThreads; base < n; base += stride) {
        const unsigned long long i = base + threadIdx.x;
        const uint32_t s = i < n ? __ldcs(slot_ids + i) : GI_SLOT_NONE;
        const bool hit = s < slots;
        if (hit) {
            Accum *a = acc + s;
            if (BITMAP) {
                bulk_wait_read();
                s_red[threadIdx.x][0] = 1ull;
                s_red[threadIdx.x][1] = 2ull;
                s_red[threadIdx.x][2] = 3ull;
                s_red[threadIdx.x][3] = 1ull;
                bulk_add_accum(a, s_red[threadIdx.x]);
                atomicOr(bitmap + (s >> 5), 1u << (s & 31u));
            } else {
                atomicAdd(&a->sum[0], 1ull);
                atomicAdd(&a->sum[1], 2ull);
                atomicAdd(&a->sum[2], 3ull);
                if (atomicAdd(&a->count, 1u) == 0u) ++first;
            }
        }
    }
    if (BITMAP) {
        bulk_wait_all();
        return;
    }
    first = __reduce_add_sync(kFull, first);
    if (lane == 0 && first) atomicAdd(&s_first, first);
    __syncthreads();
    if (threadIdx.x == 0 && s_first) atomicAdd(first_out, s_first);
}

} // namespace gi

using namespace gi;

extern "C" gi_status gi_diag_update_atomics(const uint32_t *slot_ids, uint64_t n, uint32_t log2_slots,
                                            uint32_t first_touch, void *scratch, uint32_t *first_touches,
                                            gi_stream_t stream) {
    if (log2_slots < 10 || log2_slots > 30) {
        set_error("gi_diag_update_atomics: log2_slots must be in [10, 30]");
        return GI_ERR_INVALID_ARG;
    }
    if (first_touch > GI_FIRST_TOUCH_BITMAP) {
        set_error("gi_diag_update_atomics: unknown first_touch form");
        return GI_ERR_INVALID_ARG;
    }
    const bool bitmap = first_touch != GI_FIRST_TOUCH_LIST;
    if ((n > 0 && !slot_ids) || !scratch || (!bitmap && !first_touches)) {
        set_error("gi_diag_update_atomics: NULL buffer");
        return GI_ERR_INVALID_ARG;
    }
    if ((reinterpret_cast<uintptr_t>(scratch) & 31u) != 0 || (reinterpret_cast<uintptr_t>(first_touches) & 3u) != 0 ||
        (reinterpret_cast<uintptr_t>(slot_ids) & 3u) != 0) {
        set_error("gi_diag_update_atomics: scratch must be 32-byte aligned, slot_ids and first_touches 4-byte aligned");
        return GI_ERR_INVALID_ARG;
    }
    if (n == 0) return GI_OK;
    const uint32_t slots = 1u << log2_slots;
    Accum *acc = static_cast<Accum *>(scratch);
    uint32_t *bits = reinterpret_cast<uint32_t *>(acc + slots);
    const unsigned blocks = (unsigned)((n + kUpdBlockRecords - 1) / kUpdBlockRecords);
    cudaStream_t st = (cudaStream_t)stream;
    if (bitmap)
        k_diag_atomics<true><<<blocks, kUpdThreads, 0, st>>>(slot_ids, (unsigned long long)n, slots, acc, bits, nullptr);
    else
        k_diag_atomics<false><<<blocks, kUpdThreads, 0, st>>>(slot_ids, (unsigned long long)n, slots, acc, nullptr,
                                                              first_touches);
    return cuda_status(cudaGetLastError(), "k_diag_atomics launch");
}
