// Learned radiance surrogate: multiresolution hash encoding (Mueller et al. 2022) of the hit
// position and normal direction code, a 32 -> 64 -> 64 -> 3 ReLU network without bias terms on the
// fifth-generation tensor cores (tcgen05 MMAs from shared memory into tensor memory), relative-L2
// loss (Mueller et al. 2021) and Adam (Kingma and Ba 2015), trained online on the world cache's
// resolved cells.  The paper itself has no learned part.
//
// Passes of one training step (all on the caller's stream):
//   k_nrc_encode   one thread per (sample, level): normalise the position, find the level's cell,
//                  gather the 8 vertices' float16 features, interpolate, write the sample's row of
//                  the bf16 input tile (and its target / mask plane, and record index)
//   k_nrc_mlp      persistent, one CTA per SM, 128-sample tiles: forward, loss gradient, backward
//                  through the three layers, weight gradients accumulated in tensor memory over all
//                  the CTA's tiles, input gradients out to global memory
//   k_nrc_scatter  one thread per (sample, level): trilinear weights x input gradient added to the
//                  8 vertices' gradient accumulators (float2 atomics)
//   k_nrc_adam_*   Adam on the table entries and the weights; refreshes the float16 table copy and
//                  the bf16 weight images the MLP kernel loads
//
// Shared-memory operand layout: see gi_tc.cuh (K-major core matrices, no swizzle).  Every tile of
// the MLP kernel is stored sample-major; the weight-gradient products, which contract over the
// samples, read the same tiles through MN-major descriptors (LBO = stride between 8-sample groups,
// SBO = stride between 8-feature groups), so no tile is ever transposed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <vector>

#include "gi_internal.cuh"
#include "gi_tc.cuh"

namespace gi {
namespace {

constexpr int kL = GI_NRC_LEVELS;    // 16 levels
constexpr int kIn = 2 * kL;          // 32 encoded features
constexpr int kHid = GI_NRC_HIDDEN;  // 64 hidden units
constexpr int kOut = GI_NRC_OUTPUTS; // 3 outputs
constexpr int kTile = 128;           // samples per tile = M of every forward / backward product
constexpr int kEncThreads = 256;
constexpr uint32_t kPrimeY = 2654435761u, kPrimeZ = 805459861u, kPrimeD = 2246822519u;

// bf16 weight images (core-matrix tiles), loaded into shared memory by every MLP CTA
constexpr uint32_t kImgW1 = 0;        // W1   [64 out][32 in]   SBO 512
constexpr uint32_t kImgW1T = 4096;    // W1^T [32 in][64 out]   SBO 1024
constexpr uint32_t kImgW2 = 8192;     // W2   [64][64]          SBO 1024
constexpr uint32_t kImgW2T = 16384;   // W2^T [64][64]          SBO 1024
constexpr uint32_t kImgW3P = 24576;   // W3   [16 out][64 in]   SBO 1024, rows 3..15 zero
constexpr uint32_t kImgW3PT = 26624;  // W3^T [64 in][16 out]   SBO 256, columns 3..15 zero
constexpr uint32_t kImgBytes = 28672;

// float32 master weights: W1 | W2 | W3, row-major [out][in]
constexpr int kW1 = 0, kW2 = kHid * kIn, kW3 = kW2 + kHid * kHid, kWCount = kW3 + kOut * kHid;
// a CTA's partial: the weight gradients of its tiles, then its loss, sum m|y - t|, sum m|t|
constexpr int kPartStride = kWCount + 4;

// global input tile: [128 samples][32 features] bf16 core matrices; 8-sample group g = bytes 512 g ..
constexpr uint32_t kXTile = kTile * kIn * 2;  // 8192
constexpr uint32_t kTTile = 4 * kTile * 4;    // target planes r, g, b and the mask: 2048

// MLP kernel shared memory (bytes)
constexpr uint32_t kSmImg = 0;
constexpr uint32_t kSmXH0 = 28672;   // [128][96]: H1 (features 0..63) | X (64..95), SBO 1536
constexpr uint32_t kSmXH1 = 53248;
constexpr uint32_t kSmT0 = 77824;    // target tiles
constexpr uint32_t kSmT1 = 79872;
constexpr uint32_t kSmH2 = 81920;    // [128][64], SBO 1024
constexpr uint32_t kSmDY = 98304;    // [128][16], SBO 256
constexpr uint32_t kSmZ = 102400;    // [128][128]: dZ2 (0..63) | dZ1 (64..127), SBO 2048
constexpr uint32_t kSmTrain = 135168;
constexpr uint32_t kSmInfer = 98304; // image, XH0, XH1, (targets unused), H2
constexpr uint32_t kXHStride = 1536, kH2Stride = 1024, kDYStride = 256, kZStride = 2048;

// tensor memory columns (256 allocated)
constexpr uint32_t kTmD1 = 0;    // layer-1 pre-activation, then dH1, then dX
constexpr uint32_t kTmD2 = 64;   // layer-2 pre-activation, then dH2
constexpr uint32_t kTmD3 = 128;  // output (16 columns, 3 used)
constexpr uint32_t kTmGC = 144;  // dW3^T accumulator (16 columns)
constexpr uint32_t kTmGA = 160;  // [dW2 | dW1] accumulator (96 columns)
constexpr uint32_t kTmCols = 256;

constexpr uint32_t kErrTimeout = 1u;

// One table entry: float32 master features and Adam moments, padded to one sector.  The
// gradient accumulators live in a separate dense float2 array, so that the Adam pass can find
// the entries a step touched with one coalesced 8-byte read per entry.
struct __align__(32) Entry {
    float2 p, m, v, pad;
};
static_assert(sizeof(Entry) == 32, "entry must fill one sector");

struct Levels {
    uint32_t res[kL];
    uint32_t dense[kL];
};

struct Geometry {
    float lo[3], inv_ext[3];
    Levels lv;
    uint32_t log2_table;
};

enum EncMode { kEncPoints = 0, kEncSampled = 1, kEncQueries = 2 };

struct EncArgs {
    Geometry geo;
    const __half2 *tab16;
    // points (mode kEncPoints) or records (modes kEncSampled, kEncQueries)
    const float *pos[3];
    const float *nrm[3];
    const float *len;          // records: ray length (hit test)
    uint32_t n;                // samples (points / batch); queries: capacity
    const float *target[3];    // kEncPoints training targets (or NULL)
    const float *mask;         // kEncPoints sample mask (or NULL = 1)
    // kEncSampled: sample s of the launch is sample offset + s of the frame
    uint32_t n_records, seed, offset;
    const uint32_t *slot_ids;
    CacheView cv;
    // kEncQueries
    const uint32_t *qidx;
    const uint32_t *qcount;
    // outputs
    uint16_t *X;               // input tiles
    float *T;                  // target tiles (NULL when not training)
    uint32_t *idx;             // record index per sample (kEncSampled)
};

struct MlpArgs {
    const uint16_t *X;
    const float *T;
    const uint8_t *wimg;
    uint32_t n;                // samples, unless count is given
    const uint32_t *count;     // device sample count (queries), clamped to n
    float dy_scale;            // 2 / B
    float loss_eps;
    float *dX;                 // train: [n_pad][32] float32
    float *wpart;              // train: per-CTA partial W1 | W2 | W3 gradients and loss sums,
                               // rows of kPartStride floats (reduced by k_nrc_wgrad_reduce)
    float4 *out;               // infer: (max(y, 0), 1)
    const uint32_t *out_idx;   // infer: out[out_idx[s]] when given, else out[s]
    uint32_t *err;
};

struct ScatterArgs {
    Geometry geo;
    const float *pos[3];
    const float *nrm[3];
    const uint32_t *idx;       // record of each sample (NULL: sample s is point s)
    uint32_t n;
    const float *dX;
    float2 *grad;
};

struct SelectArgs {
    const float *pos[3];
    const float *len;
    const uint32_t *slot_ids;
    uint32_t n;
    CacheView cv;
    KeyParams kp;
    uint32_t query_lod;
    float trust;
    uint32_t trained;
    const float *stats;
    uint32_t max_q;
    uint32_t *qidx;
    uint32_t *qcount;
    uint32_t *bits;
};

// ---------------------------------------------------------------- encoding

// dominant axis of the normal (ties x, then y) and the sign bit of that component
__device__ __forceinline__ uint32_t dir_code(float nx, float ny, float nz) {
    const float ax = fabsf(nx), ay = fabsf(ny), az = fabsf(nz);
    const int axis = (ax >= ay && ax >= az) ? 0 : (ay >= az ? 1 : 2);
    const float comp = axis == 0 ? nx : (axis == 1 ? ny : nz);
    return 2u * (uint32_t)axis + (__float_as_uint(comp) >> 31);
}

// Table indices (within the level) and trilinear weights of the 8 vertices around a point.
// Corner c has offsets (c & 1, c >> 1 & 1, c >> 2 & 1).  x: normalised position in [0, 1]^3.
__device__ __forceinline__ void level_corners(const float (&x)[3], uint32_t R, bool dense, uint32_t d,
                                              uint32_t tmask, uint32_t (&idx)[8], float (&w)[8]) {
    uint32_t i[3];
    float f[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float s = __fmul_rn(x[a], (float)R);
        const int ii = min(__float2int_rd(s), (int)R - 1);
        i[a] = (uint32_t)ii;
        f[a] = __fsub_rn(s, (float)ii);
    }
    const uint32_t V = R + 1u;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        const uint32_t vx = i[0] + (c & 1), vy = i[1] + ((c >> 1) & 1), vz = i[2] + ((c >> 2) & 1);
        idx[c] = dense ? ((d * V + vz) * V + vy) * V + vx : ((vx ^ (vy * kPrimeY) ^ (vz * kPrimeZ) ^ (d * kPrimeD)) & tmask);
        const float wx = (c & 1) ? f[0] : 1.0f - f[0];
        const float wy = ((c >> 1) & 1) ? f[1] : 1.0f - f[1];
        const float wz = ((c >> 2) & 1) ? f[2] : 1.0f - f[2];
        w[c] = wx * wy * wz;
    }
}

__device__ __forceinline__ void normalise(const Geometry &g, float px, float py, float pz, float (&x)[3]) {
    const float p[3] = {px, py, pz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // fmaxf turns NaN into 0
        x[a] = fminf(fmaxf(__fmul_rn(__fsub_rn(p[a], g.lo[a]), g.inv_ext[a]), 0.0f), 1.0f);
    }
}

__device__ __forceinline__ bool record_hit(const float *const pos[3], const float *len, uint32_t r) {
    const float l = __ldg(len + r);
    return isfinite(l) && l >= 0.0f && isfinite(__ldg(pos[0] + r)) && isfinite(__ldg(pos[1] + r)) &&
           isfinite(__ldg(pos[2] + r));
}

__device__ __forceinline__ float4 cache_value(const CacheView &cv, uint32_t s) {
    const char *r = static_cast<const char *>(cv.resolved) + (size_t)s * cv.resolved_stride;
    if (cv.resolved_f16) {
        const ushort4 h = __ldg(reinterpret_cast<const ushort4 *>(r));
        return make_float4(__half2float(__ushort_as_half(h.x)), __half2float(__ushort_as_half(h.y)),
                           __half2float(__ushort_as_half(h.z)), __half2float(__ushort_as_half(h.w)));
    }
    return __ldg(reinterpret_cast<const float4 *>(r));
}

template <int MODE>
__global__ void __launch_bounds__(kEncThreads) k_nrc_encode(EncArgs a) {
    uint32_t n = a.n;
    if (MODE == kEncQueries) n = min(__ldg(a.qcount), a.n);
    const uint32_t n_pad = (n + kTile - 1) / kTile * kTile;
    const uint32_t T = 1u << a.geo.log2_table;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad * kL; i += gridDim.x * blockDim.x) {
        const uint32_t s = i >> 4, l = i & 15u;
        const bool valid = s < n;
        uint32_t r = s;
        if (MODE == kEncSampled) r = pcg_hash((a.offset + s) ^ a.seed) % a.n_records;
        if (MODE == kEncQueries && valid) r = __ldg(a.qidx + s);
        float e0 = 0.0f, e1 = 0.0f;
        if (valid) {
            float x[3];
            normalise(a.geo, __ldg(a.pos[0] + r), __ldg(a.pos[1] + r), __ldg(a.pos[2] + r), x);
            const uint32_t d = dir_code(__ldg(a.nrm[0] + r), __ldg(a.nrm[1] + r), __ldg(a.nrm[2] + r));
            uint32_t idx[8];
            float w[8];
            level_corners(x, a.geo.lv.res[l], a.geo.lv.dense[l] != 0u, d, T - 1u, idx, w);
            const __half2 *tab = a.tab16 + (size_t)l * T;
            __half2 f[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) f[c] = __ldg(tab + idx[c]);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                const float2 v = __half22float2(f[c]);
                e0 = fmaf(w[c], v.x, e0);
                e1 = fmaf(w[c], v.y, e1);
            }
        }
        const uint32_t tile = s / kTile, row = s % kTile;
        uint8_t *xt = reinterpret_cast<uint8_t *>(a.X) + (size_t)tile * kXTile;
        *reinterpret_cast<__nv_bfloat162 *>(xt + tc::cm_offset(row, 2u * l, kIn)) = __floats2bfloat162_rn(e0, e1);
        if (MODE != kEncQueries && a.T && l == 0) {
            float t[3] = {0.f, 0.f, 0.f}, m = 0.0f;
            if (valid && MODE == kEncPoints) {
                for (int c = 0; c < 3; ++c) t[c] = __ldg(a.target[c] + s);
                m = a.mask ? __ldg(a.mask + s) : 1.0f;
            }
            if (valid && MODE == kEncSampled) {
                const uint32_t slot = __ldg(a.slot_ids + r);
                if (slot < a.cv.slots && record_hit(a.pos, a.len, r)) {
                    const float4 v = cache_value(a.cv, slot);
                    t[0] = v.x;
                    t[1] = v.y;
                    t[2] = v.z;
                    m = 1.0f;
                }
                a.idx[s] = r;
            }
            float *tt = a.T + (size_t)tile * (kTTile / 4);
            for (int c = 0; c < 3; ++c) tt[c * kTile + row] = t[c];
            tt[3 * kTile + row] = m;
        }
    }
}

// ---------------------------------------------------------------- the network on the tensor cores

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t *>(&h);
}

// Store 8 consecutive features (k0 .. k0 + 7) of sample row t as one 16-byte core-matrix row.
__device__ __forceinline__ void store_row8(uint8_t *tile, uint32_t row_stride, uint32_t t, uint32_t k0, const float *v) {
    const uint4 q = make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                               pack_bf16x2(v[6], v[7]));
    *reinterpret_cast<uint4 *>(tile + (t >> 3) * row_stride + (k0 >> 3) * 128u + (t & 7u) * 16u) = q;
}

// 64 accumulator columns of this thread's row
__device__ __forceinline__ void tmem_ld64(uint32_t tmem, uint32_t warp, uint32_t col, float (&z)[64]) {
    float v0[16], v1[16], v2[16], v3[16];
    tc::tmem_ld16(tc::tmem_lane_addr(tmem, warp, col), v0);
    tc::tmem_ld16(tc::tmem_lane_addr(tmem, warp, col + 16), v1);
    tc::tmem_ld16(tc::tmem_lane_addr(tmem, warp, col + 32), v2);
    tc::tmem_ld16(tc::tmem_lane_addr(tmem, warp, col + 48), v3);
    tc::wait_ld();
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        z[j] = v0[j];
        z[16 + j] = v1[j];
        z[32 + j] = v2[j];
        z[48 + j] = v3[j];
    }
}

__device__ __forceinline__ uint32_t idesc_mn(uint32_t M, uint32_t N) {
    return tc::idesc_bf16(M, N) | (1u << 15) | (1u << 16);
}

// Persistent kernel: CTA b takes tiles b, b + gridDim.x, ...; thread t owns sample row t of a tile
// (tensor-memory lane t: warp w reads lanes 32 w .. 32 w + 31).  Thread 0 issues every MMA and
// bulk copy; completion comes back through mbarriers, every wait bounded in time.
template <bool TRAIN>
__global__ void __launch_bounds__(kTile, TRAIN ? 1 : 2) k_nrc_mlp(MlpArgs a) {
    extern __shared__ __align__(1024) uint8_t smem[];
    __shared__ __align__(8) uint64_t bar_w, bar_ld[2], bar_mma;
    __shared__ uint32_t tmem_s;
    __shared__ int abort_s;
    const uint32_t t = threadIdx.x, warp = t >> 5;
    uint32_t n = a.n;
    if (a.count) n = min(__ldg(a.count), a.n);
    const uint32_t tiles = (n + kTile - 1) / kTile;
    if (blockIdx.x >= tiles) return;

    if (t == 0) {
        abort_s = 0;
        tc::mbar_init(&bar_w, 1);
        tc::mbar_init(&bar_ld[0], 1);
        tc::mbar_init(&bar_ld[1], 1);
        tc::mbar_init(&bar_mma, 1);
        tc::mbar_init_fence();
    }
    if (TRAIN) {
        // dY columns 3..15 stay zero; written once here, never again
        for (uint32_t i = t; i < kTile * 16 / 8; i += kTile)
            reinterpret_cast<uint4 *>(smem + kSmDY)[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    if (warp == 0) {
        tc::tmem_alloc(&tmem_s, kTmCols);
        tc::tmem_relinquish();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = tmem_s;
    const uint32_t sm = tc::smem_u32(smem);
    auto xh_off = [](int buf) { return buf ? kSmXH1 : kSmXH0; };
    auto t_off = [](int buf) { return buf ? kSmT1 : kSmT0; };
    // Thread 0 counts the asynchronous operations it started and the completions it saw, so that
    // a CTA that gives up after a wait ran out first waits (bounded again) for what it still has in
    // flight -- at most one load per buffer and one MMA group -- before freeing its tensor memory.
    uint32_t ld_issued[2] = {0u, 0u}, ld_done[2] = {0u, 0u}, mma_issued = 0u, mma_done = 0u;
    bool w_done = false;

    auto load_tile = [&](uint32_t tile, int buf) {  // thread 0 only
        ++ld_issued[buf];
        const uint32_t bytes = kXTile + (TRAIN ? kTTile : 0u);
        tc::mbar_expect_tx(&bar_ld[buf], bytes);
        const uint8_t *src = reinterpret_cast<const uint8_t *>(a.X) + (size_t)tile * kXTile;
        for (uint32_t g = 0; g < kTile / 8; ++g)
            tc::bulk_g2s(smem + xh_off(buf) + g * kXHStride + 1024u, src + g * 512u, 512u, &bar_ld[buf]);
        if (TRAIN)
            tc::bulk_g2s(smem + t_off(buf), reinterpret_cast<const uint8_t *>(a.T) + (size_t)tile * kTTile, kTTile,
                         &bar_ld[buf]);
    };
    if (t == 0) {
        tc::mbar_expect_tx(&bar_w, kImgBytes);
        tc::bulk_g2s(smem + kSmImg, a.wimg, kImgBytes, &bar_w);
        load_tile(blockIdx.x, 0);
    }
    bool ok = tc::mbar_wait(&bar_w, 0);
    w_done = ok;
    uint32_t ph = 0;  // parity of the next MMA completion
    float loss = 0.f, jerr = 0.f, jtgt = 0.f;
    uint32_t it = 0;
    auto commit_mma = [&]() {  // thread 0 only
        tc::commit(&bar_mma);
        ++mma_issued;
    };
    auto mma_wait = [&]() {
        const bool got = tc::mbar_wait(&bar_mma, ph);
        if (got) ++mma_done;
        ok = got && ok;
        ph ^= 1u;
        tc::fence_after_sync();
    };
    auto sync_operands = [&]() {  // generic smem writes -> tensor cores; TMEM reads done
        tc::fence_async_smem();
        tc::fence_before_sync();
        if (!ok) abort_s = 1;
        __syncthreads();
    };

    for (uint32_t tile = blockIdx.x; tile < tiles; tile += gridDim.x, ++it) {
        const int buf = it & 1;
        const bool got = tc::mbar_wait(&bar_ld[buf], (it >> 1) & 1u);
        if (got) ++ld_done[buf];
        ok = got && ok;
        if (!ok) abort_s = 1;
        __syncthreads();
        if (abort_s) break;
        if (t == 0 && tile + gridDim.x < tiles) load_tile(tile + gridDim.x, buf ^ 1);
        const uint32_t xh = sm + xh_off(buf);
        uint8_t *xh_p = smem + xh_off(buf);

        // ---- layer 1: D1 = X W1^T
        if (t == 0) {
            tc::fence_after_sync();
            for (uint32_t ks = 0; ks < kIn / 16; ++ks)
                tc::mma_bf16(tmem + kTmD1, tc::smem_desc(xh + 1024u + ks * 256u, 128u, kXHStride),
                             tc::smem_desc(sm + kSmImg + kImgW1 + ks * 256u, 128u, 512u), tc::idesc_bf16(128, 64), ks);
            commit_mma();
        }
        mma_wait();
        float z[64];
        uint32_t m1[2] = {0u, 0u}, m2[2] = {0u, 0u};
        tmem_ld64(tmem, warp, kTmD1, z);
#pragma unroll
        for (int j = 0; j < 64; ++j) {
            m1[j >> 5] |= (z[j] > 0.0f ? 1u : 0u) << (j & 31);
            z[j] = fmaxf(z[j], 0.0f);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) store_row8(xh_p, kXHStride, t, 8u * j, z + 8 * j);
        sync_operands();
        if (abort_s) break;

        // ---- layer 2: D2 = H1 W2^T
        if (t == 0) {
            tc::fence_after_sync();
            for (uint32_t ks = 0; ks < kHid / 16; ++ks)
                tc::mma_bf16(tmem + kTmD2, tc::smem_desc(xh + ks * 256u, 128u, kXHStride),
                             tc::smem_desc(sm + kSmImg + kImgW2 + ks * 256u, 128u, 1024u), tc::idesc_bf16(128, 64), ks);
            commit_mma();
        }
        mma_wait();
        tmem_ld64(tmem, warp, kTmD2, z);
#pragma unroll
        for (int j = 0; j < 64; ++j) {
            m2[j >> 5] |= (z[j] > 0.0f ? 1u : 0u) << (j & 31);
            z[j] = fmaxf(z[j], 0.0f);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) store_row8(smem + kSmH2, kH2Stride, t, 8u * j, z + 8 * j);
        sync_operands();
        if (abort_s) break;

        // ---- layer 3: D3 = H2 W3^T (16 columns, 3 used)
        if (t == 0) {
            tc::fence_after_sync();
            for (uint32_t ks = 0; ks < kHid / 16; ++ks)
                tc::mma_bf16(tmem + kTmD3, tc::smem_desc(sm + kSmH2 + ks * 256u, 128u, kH2Stride),
                             tc::smem_desc(sm + kSmImg + kImgW3P + ks * 256u, 128u, 1024u), tc::idesc_bf16(128, 16), ks);
            commit_mma();
        }
        mma_wait();
        float y[16];
        tc::tmem_ld16(tc::tmem_lane_addr(tmem, warp, kTmD3), y);
        tc::wait_ld();
        const uint32_t s = tile * kTile + t;

        if (!TRAIN) {
            if (s < n) {
                const uint32_t o = a.out_idx ? __ldg(a.out_idx + s) : s;
                a.out[o] = make_float4(fmaxf(y[0], 0.0f), fmaxf(y[1], 0.0f), fmaxf(y[2], 0.0f), 1.0f);
            }
            tc::fence_before_sync();
            __syncthreads();  // the next tile's products overwrite the accumulators just read
            continue;
        }

        // ---- loss gradient: dy = m (2 / B) (y - t) / (y^2 + eps); relative L2 and the judge's sums
        const float *tt = reinterpret_cast<const float *>(smem + t_off(buf));
        const float msk = tt[3 * kTile + t];
        float dy[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int c = 0; c < kOut; ++c) {
            const float tg = tt[c * kTile + t];
            const float r = y[c] - tg;
            const float den = y[c] * y[c] + a.loss_eps;
            dy[c] = msk * a.dy_scale * r / den;
            loss += msk * r * r / den;
            jerr += msk * fabsf(r);
            jtgt += msk * fabsf(tg);
        }
        {
            const float zero8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
            store_row8(smem + kSmDY, kDYStride, t, 0u, dy);
            store_row8(smem + kSmDY, kDYStride, t, 8u, zero8);
        }
        sync_operands();
        if (abort_s) break;

        // ---- dH2 = dY W3 (K = 16)
        if (t == 0) {
            tc::fence_after_sync();
            tc::mma_bf16(tmem + kTmD2, tc::smem_desc(sm + kSmDY, 128u, kDYStride),
                         tc::smem_desc(sm + kSmImg + kImgW3PT, 128u, 256u), tc::idesc_bf16(128, 64), 0u);
            commit_mma();
        }
        mma_wait();
        tmem_ld64(tmem, warp, kTmD2, z);
#pragma unroll
        for (int j = 0; j < 64; ++j) z[j] = ((m2[j >> 5] >> (j & 31)) & 1u) ? z[j] : 0.0f;
#pragma unroll
        for (int j = 0; j < 8; ++j) store_row8(smem + kSmZ, kZStride, t, 8u * j, z + 8 * j);
        sync_operands();
        if (abort_s) break;

        // ---- dH1 = dZ2 W2
        if (t == 0) {
            tc::fence_after_sync();
            for (uint32_t ks = 0; ks < kHid / 16; ++ks)
                tc::mma_bf16(tmem + kTmD1, tc::smem_desc(sm + kSmZ + ks * 256u, 128u, kZStride),
                             tc::smem_desc(sm + kSmImg + kImgW2T + ks * 256u, 128u, 1024u), tc::idesc_bf16(128, 64), ks);
            commit_mma();
        }
        mma_wait();
        tmem_ld64(tmem, warp, kTmD1, z);
#pragma unroll
        for (int j = 0; j < 64; ++j) z[j] = ((m1[j >> 5] >> (j & 31)) & 1u) ? z[j] : 0.0f;
#pragma unroll
        for (int j = 0; j < 8; ++j) store_row8(smem + kSmZ, kZStride, t, 64u + 8u * j, z + 8 * j);
        sync_operands();
        if (abort_s) break;

        // ---- dX = dZ1 W1; weight gradients over the tile's samples (MN-major operands):
        //      [dW2 | dW1] += [dZ2 | dZ1]^T [H1 | X],  dW3^T += H2^T dY
        if (t == 0) {
            tc::fence_after_sync();
            for (uint32_t ks = 0; ks < kHid / 16; ++ks)
                tc::mma_bf16(tmem + kTmD1, tc::smem_desc(sm + kSmZ + 1024u + ks * 256u, 128u, kZStride),
                             tc::smem_desc(sm + kSmImg + kImgW1T + ks * 256u, 128u, 1024u), tc::idesc_bf16(128, 32), ks);
            for (uint32_t ks = 0; ks < kTile / 16; ++ks)
                tc::mma_bf16(tmem + kTmGA, tc::smem_desc(sm + kSmZ + ks * 2u * kZStride, kZStride, 128u),
                             tc::smem_desc(xh + ks * 2u * kXHStride, kXHStride, 128u), idesc_mn(128, 96),
                             (it | ks) != 0u);
            // rows 64..127 of this A operand run past H2 into the dY tile: they only feed
            // accumulator rows that are never read
            for (uint32_t ks = 0; ks < kTile / 16; ++ks)
                tc::mma_bf16(tmem + kTmGC, tc::smem_desc(sm + kSmH2 + ks * 2u * kH2Stride, kH2Stride, 128u),
                             tc::smem_desc(sm + kSmDY + ks * 2u * kDYStride, kDYStride, 128u), idesc_mn(128, 16),
                             (it | ks) != 0u);
            commit_mma();
        }
        mma_wait();
        {
            float g0[16], g1[16];
            tc::tmem_ld16(tc::tmem_lane_addr(tmem, warp, kTmD1), g0);
            tc::tmem_ld16(tc::tmem_lane_addr(tmem, warp, kTmD1 + 16), g1);
            tc::wait_ld();
            float4 *dst = reinterpret_cast<float4 *>(a.dX + (size_t)s * kIn);
#pragma unroll
            for (int j = 0; j < 4; ++j) dst[j] = make_float4(g0[4 * j], g0[4 * j + 1], g0[4 * j + 2], g0[4 * j + 3]);
#pragma unroll
            for (int j = 0; j < 4; ++j) dst[4 + j] = make_float4(g1[4 * j], g1[4 * j + 1], g1[4 * j + 2], g1[4 * j + 3]);
        }
        tc::fence_before_sync();
        if (!ok) abort_s = 1;
        __syncthreads();
        if (abort_s) break;
    }

    float *part = TRAIN ? a.wpart + (size_t)blockIdx.x * kPartStride : nullptr;
    if (abort_s) {
        if (t == 0) {
            atomicOr(a.err, kErrTimeout);
            // what thread 0 started and has not seen complete: the weight image, one load per
            // buffer, one MMA group (a buffer is reloaded, and an MMA group committed, only after
            // the previous one was waited for, so each barrier has at most one phase pending)
            if (!w_done) tc::mbar_wait(&bar_w, 0);
            for (int b = 0; b < 2; ++b)
                if (ld_issued[b] > ld_done[b]) tc::mbar_wait(&bar_ld[b], (ld_issued[b] - 1u) & 1u);
            if (mma_issued > mma_done) tc::mbar_wait(&bar_mma, (mma_issued - 1u) & 1u);
        }
        if (TRAIN)
            for (int i = t; i < kPartStride; i += kTile) part[i] = 0.0f;
    } else if (TRAIN && it > 0) {
        // weight gradients of this CTA's tiles: rows 0..63 of GA are dW2, rows 64..127 columns
        // 64..95 are dW1; rows 0..63 of GC are dW3^T.  Plain stores into the CTA's partial row.
        tc::fence_after_sync();
        if (warp < 2) {
            float z[64];
            tmem_ld64(tmem, warp, kTmGA, z);
            float4 *d2 = reinterpret_cast<float4 *>(part + kW2 + t * kHid);
#pragma unroll
            for (int j = 0; j < 16; ++j) d2[j] = make_float4(z[4 * j], z[4 * j + 1], z[4 * j + 2], z[4 * j + 3]);
            float g[16];
            tc::tmem_ld16(tc::tmem_lane_addr(tmem, warp, kTmGC), g);
            tc::wait_ld();
            for (int c = 0; c < kOut; ++c) part[kW3 + c * kHid + t] = g[c];
        } else {
            float g0[16], g1[16];
            tc::tmem_ld16(tc::tmem_lane_addr(tmem, warp, kTmGA + 64), g0);
            tc::tmem_ld16(tc::tmem_lane_addr(tmem, warp, kTmGA + 80), g1);
            tc::wait_ld();
            float4 *d1 = reinterpret_cast<float4 *>(part + kW1 + (t - 64) * kIn);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                d1[j] = make_float4(g0[4 * j], g0[4 * j + 1], g0[4 * j + 2], g0[4 * j + 3]);
                d1[4 + j] = make_float4(g1[4 * j], g1[4 * j + 1], g1[4 * j + 2], g1[4 * j + 3]);
            }
        }
        for (int d = 16; d; d >>= 1) {
            loss += __shfl_xor_sync(0xFFFFFFFFu, loss, d);
            jerr += __shfl_xor_sync(0xFFFFFFFFu, jerr, d);
            jtgt += __shfl_xor_sync(0xFFFFFFFFu, jtgt, d);
        }
        __shared__ float red_s[4][3];
        if ((t & 31) == 0) {
            red_s[warp][0] = loss;
            red_s[warp][1] = jerr;
            red_s[warp][2] = jtgt;
        }
        __syncthreads();
        if (t < 3) part[kWCount + t] = (red_s[0][t] + red_s[1][t] + red_s[2][t] + red_s[3][t]) * (t == 0 ? 0.5f * a.dy_scale : 1.0f);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, kTmCols);
}

// ---------------------------------------------------------------- gradient scatter and Adam

// Sum the MLP kernel's per-CTA partials into the weight-gradient accumulators and the loss sums.
// Block = 32 consecutive values x 8 warps; warp w sums parts w, w + 8, ...; then the 8 warp sums
// in a fixed order (deterministic).
__global__ void __launch_bounds__(256) k_nrc_wgrad_reduce(const float *wpart, int parts, float *wg, float *stats) {
    __shared__ float acc[8][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int i = blockIdx.x * 32 + lane;
    float s = 0.0f;
    if (i < kWCount + 3) {
#pragma unroll 4
        for (int p = w; p < parts; p += 8) s += __ldcg(wpart + (size_t)p * kPartStride + i);
    }
    acc[w][lane] = s;
    __syncthreads();
    if (w == 0 && i < kWCount + 3) {
        float t = 0.0f;
#pragma unroll
        for (int k = 0; k < 8; ++k) t += acc[k][lane];
        if (i < kWCount) wg[i] += t;
        else stats[i - kWCount] += t;
    }
}

__global__ void __launch_bounds__(kEncThreads) k_nrc_scatter(ScatterArgs a) {
    const uint32_t T = 1u << a.geo.log2_table;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < a.n * kL; i += gridDim.x * blockDim.x) {
        const uint32_t s = i >> 4, l = i & 15u;
        const float2 g = __ldg(reinterpret_cast<const float2 *>(a.dX + (size_t)s * kIn) + l);
        if (g.x == 0.0f && g.y == 0.0f) continue;
        const uint32_t r = a.idx ? __ldg(a.idx + s) : s;
        float x[3];
        normalise(a.geo, __ldg(a.pos[0] + r), __ldg(a.pos[1] + r), __ldg(a.pos[2] + r), x);
        const uint32_t d = dir_code(__ldg(a.nrm[0] + r), __ldg(a.nrm[1] + r), __ldg(a.nrm[2] + r));
        uint32_t idx[8];
        float w[8];
        level_corners(x, a.geo.lv.res[l], a.geo.lv.dense[l] != 0u, d, T - 1u, idx, w);
        float2 *gt = a.grad + (size_t)l * T;
#pragma unroll
        for (int c = 0; c < 8; ++c) atomicAdd(gt + idx[c], make_float2(w[c] * g.x, w[c] * g.y));
    }
}

struct AdamArgs {
    float lr, b1, b2, eps, c1, c2;  // c1 = 1 - b1^t, c2 = 1 - b2^t
};

__device__ __forceinline__ float adam_update(float p, float &m, float &v, float g, const AdamArgs &a) {
    m = a.b1 * m + (1.0f - a.b1) * g;
    v = a.b2 * v + (1.0f - a.b2) * g * g;
    return p - a.lr * (m / a.c1) / (sqrtf(v / a.c2) + a.eps);
}

// Sparse Adam on the table: an entry whose gradient is (0, 0) this step keeps its value and its
// moments (the samples of the step did not touch it); the others take an Adam step with the
// global step count's bias correction.  Gradients are cleared as they are consumed.  A thread
// takes 4 consecutive entries: one 32-byte gradient read, then the touched entries' loads issued
// together before any is used.  total is a multiple of 4.
__global__ void __launch_bounds__(256) k_nrc_adam_table(Entry *tab, float2 *grad, __half2 *tab16, uint64_t total,
                                                        AdamArgs a) {
    const uint64_t groups = total >> 2;
    for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < groups;
         q += (uint64_t)gridDim.x * blockDim.x) {
        float4 *gq = reinterpret_cast<float4 *>(grad) + 2 * q;
        const float4 g01 = gq[0], g23 = gq[1];
        const float2 g[4] = {make_float2(g01.x, g01.y), make_float2(g01.z, g01.w), make_float2(g23.x, g23.y),
                             make_float2(g23.z, g23.w)};
        bool t[4];
        bool any = false;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            t[k] = g[k].x != 0.0f || g[k].y != 0.0f;
            any |= t[k];
        }
        if (!any) continue;
        Entry e[4];
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (t[k]) e[k] = tab[4 * q + k];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (!t[k]) continue;
            e[k].p.x = adam_update(e[k].p.x, e[k].m.x, e[k].v.x, g[k].x, a);
            e[k].p.y = adam_update(e[k].p.y, e[k].m.y, e[k].v.y, g[k].y, a);
            tab[4 * q + k] = e[k];
            tab16[4 * q + k] = __floats2half2_rn(e[k].p.x, e[k].p.y);
        }
        gq[0] = make_float4(0.f, 0.f, 0.f, 0.f);
        gq[1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
}

__global__ void k_nrc_table_f16(const Entry *tab, __half2 *tab16, uint64_t n) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        tab16[i] = __floats2half2_rn(tab[i].p.x, tab[i].p.y);
}

// Master features <-> a plain float2 array: mode 0 reads them out, 1 writes them, 2 clears the
// Adam moments (buf unused).
__global__ void k_nrc_table_field(Entry *tab, float2 *buf, uint64_t n, int mode) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        if (mode == 2) tab[i].m = tab[i].v = make_float2(0.0f, 0.0f);
        else if (mode == 1) tab[i].p = buf[i];
        else buf[i] = tab[i].p;
    }
}

__device__ __forceinline__ void put_bf16(uint8_t *img, uint32_t off, float v) {
    *reinterpret_cast<__nv_bfloat16 *>(img + off) = __float2bfloat16_rn(v);
}

// Adam on the weights (update != 0), then the bf16 images W, W^T of every layer.
__global__ void __launch_bounds__(256) k_nrc_adam_mlp(float *w, float *m, float *v, float *g, uint8_t *img, int update,
                                                      AdamArgs a) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kWCount; i += gridDim.x * blockDim.x) {
        float p = w[i];
        if (update) {
            float mm = m[i], vv = v[i];
            p = adam_update(p, mm, vv, g[i], a);
            m[i] = mm;
            v[i] = vv;
            g[i] = 0.0f;
            w[i] = p;
        }
        if (i < kW2) {
            const uint32_t o = i / kIn, k = i % kIn;
            put_bf16(img, kImgW1 + tc::cm_offset(o, k, kIn), p);
            put_bf16(img, kImgW1T + tc::cm_offset(k, o, kHid), p);
        } else if (i < kW3) {
            const uint32_t o = (i - kW2) / kHid, k = (i - kW2) % kHid;
            put_bf16(img, kImgW2 + tc::cm_offset(o, k, kHid), p);
            put_bf16(img, kImgW2T + tc::cm_offset(k, o, kHid), p);
        } else {
            const uint32_t o = (i - kW3) / kHid, k = (i - kW3) % kHid;
            put_bf16(img, kImgW3P + tc::cm_offset(o, k, kHid), p);
            put_bf16(img, kImgW3PT + tc::cm_offset(k, o, 16), p);
        }
    }
}

// ---------------------------------------------------------------- query selection

__global__ void __launch_bounds__(256) k_nrc_select(SelectArgs a) {
    const uint32_t lane = threadIdx.x & 31u;
    const bool trusted = a.trained && __ldg(a.stats + 2) > 0.0f && __ldg(a.stats + 1) <= a.trust * __ldg(a.stats + 2);
    const uint32_t words = (a.n + 31u) / 32u;
    const uint32_t warps = gridDim.x * (blockDim.x >> 5);
    for (uint32_t wd = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; wd < words; wd += warps) {
        const uint32_t r = wd * 32u + lane;
        bool use = false;
        if (r < a.n && record_hit(a.pos, a.len, r)) {
            const uint32_t slot = __ldg(a.slot_ids + r);
            if (slot == GI_SLOT_FAR) {
                // left out of the table by the update (gi_cache_route_far): the network is its only answer
                use = true;
            } else if (!trusted) {
            } else if (slot == GI_SLOT_NONE) {
                use = true;
            } else if (slot < a.cv.slots) {
                const bool cold = cache_value(a.cv, slot).w != 0.0f;
                use = cold || key_lod(a.kp, __ldg(a.pos[0] + r), __ldg(a.pos[1] + r), __ldg(a.pos[2] + r)) >=
                                  (int)a.query_lod;
            }
        }
        const uint32_t ball = __ballot_sync(0xFFFFFFFFu, use);
        uint32_t base = 0;
        if (lane == 0 && ball) base = atomicAdd(a.qcount, __popc(ball));
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        const uint32_t pos = base + __popc(ball & ((1u << lane) - 1u));
        use = use && pos < a.max_q;
        if (use) a.qidx[pos] = r;
        const uint32_t kept = __ballot_sync(0xFFFFFFFFu, use);
        if (lane == 0) a.bits[wd] = kept;
    }
}

__global__ void k_nrc_gather_answers(const uint32_t *qidx, const float4 *ovr, uint32_t count, uint32_t *records,
                                     float4 *rad) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) {
        const uint32_t r = qidx[i];
        records[i] = r;
        rad[i] = ovr[r];
    }
}

// ---------------------------------------------------------------- host side

uint64_t splitmix64(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double uniform01(uint64_t &s) { return (double)(splitmix64(s) >> 11) * (1.0 / 9007199254740992.0); }

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
}

}  // namespace
}  // namespace gi

struct gi_nrc_s {
    gi_nrc_config cfg;
    gi::Geometry geo;
    uint32_t T;
    gi::Entry *tab = nullptr;
    float2 *grad = nullptr;     // table gradient accumulators [levels][T]
    __half2 *tab16 = nullptr;
    float *w = nullptr, *wm = nullptr, *wv = nullptr, *wg = nullptr;
    uint8_t *wimg = nullptr;
    float *stats = nullptr;      // loss, sum m|y - t|, sum m|t|, spare
    float *wpart = nullptr;      // per-CTA partial weight gradients of the training network kernel
    uint32_t *err = nullptr;
    // per-batch scratch, capacity `cap` samples (a multiple of 128)
    uint32_t cap = 0;
    uint16_t *X = nullptr;
    float *Tt = nullptr;
    float *dX = nullptr;
    uint32_t *idx = nullptr;
    // query state
    uint32_t *bits = nullptr;
    float4 *ovr = nullptr;
    uint32_t *qidx = nullptr;
    uint32_t *qcount = nullptr;
    uint64_t last_query_n = 0;
    bool queried = false;
    uint64_t steps = 0;
    uint32_t last_minibatches = 1;
    int sms = 1;
};

using namespace gi;

namespace {

gi_status nrc_alloc(void **p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        set_error("gi_nrc: cudaMalloc of %zu bytes failed", bytes);
        return GI_ERR_OOM;
    }
    return GI_OK;
}

void nrc_free(gi_nrc_s *s) {
    void *ptrs[] = {s->tab, s->grad, s->tab16, s->w, s->wm, s->wv, s->wg, s->wimg, s->stats, s->err, s->wpart,
                    s->X, s->Tt, s->dX, s->idx, s->bits, s->ovr, s->qidx, s->qcount};
    for (void *p : ptrs)
        if (p) cudaFree(p);
}

gi_status ensure_capacity(gi_nrc_s *s, uint32_t n) {
    const uint32_t need = (n + kTile - 1) / kTile * kTile;
    if (need <= s->cap) return GI_OK;
    cudaDeviceSynchronize();
    for (void *p : {(void *)s->X, (void *)s->Tt, (void *)s->dX, (void *)s->idx})
        if (p) cudaFree(p);
    s->X = nullptr;
    s->Tt = nullptr;
    s->dX = nullptr;
    s->idx = nullptr;
    s->cap = 0;
    gi_status st = nrc_alloc((void **)&s->X, (size_t)need * kIn * 2);
    if (st == GI_OK) st = nrc_alloc((void **)&s->Tt, (size_t)need / kTile * kTTile);
    if (st == GI_OK) st = nrc_alloc((void **)&s->dX, (size_t)need * kIn * 4);
    if (st == GI_OK) st = nrc_alloc((void **)&s->idx, (size_t)need * 4);
    if (st == GI_OK) s->cap = need;
    return st;
}

bool points_ok(const gi_points *p) {
    if (!p || p->n > GI_NRC_MAX_BATCH) return false;
    if (p->n == 0) return true;
    for (int a = 0; a < 3; ++a)
        if (!p->pos[a] || !p->nrm[a]) return false;
    return true;
}

EncArgs enc_base(const gi_nrc_s *s) {
    EncArgs e;
    memset(&e, 0, sizeof(e));
    e.geo = s->geo;
    e.tab16 = s->tab16;
    e.X = s->X;
    e.T = s->Tt;
    e.idx = s->idx;
    return e;
}

unsigned enc_blocks(const gi_nrc_s *s, uint64_t work) {
    const uint64_t b = (work + kEncThreads - 1) / kEncThreads;
    const uint64_t cap = (uint64_t)s->sms * 8;
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(b, cap));
}

gi_status launch_mlp(gi_nrc_s *s, bool train, uint32_t n, const uint32_t *count, float dy_scale, float4 *out,
                     const uint32_t *out_idx, cudaStream_t st) {
    MlpArgs m;
    memset(&m, 0, sizeof(m));
    m.X = s->X;
    m.T = s->Tt;
    m.wimg = s->wimg;
    m.n = n;
    m.count = count;
    m.dy_scale = dy_scale;
    m.loss_eps = s->cfg.loss_eps;
    m.dX = s->dX;
    m.wpart = s->wpart;
    m.out = out;
    m.out_idx = out_idx;
    m.err = s->err;
    const uint32_t tiles = (n + kTile - 1) / kTile;
    if (tiles == 0) return GI_OK;
    if (train) {
        const unsigned grid = std::min<uint32_t>(tiles, (uint32_t)s->sms);
        k_nrc_mlp<true><<<grid, kTile, kSmTrain, st>>>(m);
        gi_status r = cuda_status(cudaGetLastError(), "k_nrc_mlp launch");
        if (r != GI_OK) return r;
        k_nrc_wgrad_reduce<<<(kWCount + 3 + 31) / 32, 256, 0, st>>>(s->wpart, (int)grid, s->wg, s->stats);
        return cuda_status(cudaGetLastError(), "k_nrc_wgrad_reduce launch");
    } else {
        const unsigned grid = std::min<uint32_t>(tiles, 2u * (uint32_t)s->sms);
        k_nrc_mlp<false><<<grid, kTile, kSmInfer, st>>>(m);
    }
    return cuda_status(cudaGetLastError(), "k_nrc_mlp launch");
}

gi_status scatter_and_return(gi_nrc_s *s, const float *const pos[3], const float *const nrm[3], const uint32_t *idx,
                             uint32_t n, cudaStream_t st) {
    ScatterArgs c;
    c.geo = s->geo;
    for (int a = 0; a < 3; ++a) {
        c.pos[a] = pos[a];
        c.nrm[a] = nrm[a];
    }
    c.idx = idx;
    c.n = n;
    c.dX = s->dX;
    c.grad = s->grad;
    k_nrc_scatter<<<enc_blocks(s, (uint64_t)n * kL), kEncThreads, 0, st>>>(c);
    return cuda_status(cudaGetLastError(), "k_nrc_scatter launch");
}

gi_status table_field(gi_nrc_s *s, float2 *host, bool grads, int mode) {
    const uint64_t entries = (uint64_t)kL * s->T;
    cudaError_t e = cudaSuccess;
    if (grads) {  // the gradient array is a plain float2 array already
        if (mode == 1) e = cudaMemcpy(s->grad, host, entries * sizeof(float2), cudaMemcpyHostToDevice);
        else e = cudaMemcpy(host, s->grad, entries * sizeof(float2), cudaMemcpyDeviceToHost);
        return cuda_status(e, "gi_nrc gradient transfer");
    }
    const unsigned blocks = (unsigned)std::min<uint64_t>((entries + 255) / 256, 65535);
    float2 *tmp = nullptr;
    if (mode != 2) {
        gi_status st = nrc_alloc((void **)&tmp, entries * sizeof(float2));
        if (st != GI_OK) return st;
    }
    if (mode == 1) e = cudaMemcpy(tmp, host, entries * sizeof(float2), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_nrc_table_field<<<blocks, 256>>>(s->tab, tmp, entries, mode);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess && mode == 0) e = cudaMemcpy(host, tmp, entries * sizeof(float2), cudaMemcpyDeviceToHost);
    if (tmp) cudaFree(tmp);
    return cuda_status(e, "gi_nrc table transfer");
}

gi_status copy_params(gi_nrc_s *s, const float *table, const float *w1, const float *w2, const float *w3, bool grads) {
    gi_status st = GI_OK;
    if (table) st = table_field(s, reinterpret_cast<float2 *>(const_cast<float *>(table)), grads, 1);
    float *dst = grads ? s->wg : s->w;
    cudaError_t e = cudaSuccess;
    if (st == GI_OK && w1) e = cudaMemcpy(dst + kW1, w1, sizeof(float) * kHid * kIn, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && st == GI_OK && w2) e = cudaMemcpy(dst + kW2, w2, sizeof(float) * kHid * kHid, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && st == GI_OK && w3) e = cudaMemcpy(dst + kW3, w3, sizeof(float) * kOut * kHid, cudaMemcpyHostToDevice);
    return st != GI_OK ? st : cuda_status(e, "gi_nrc parameter upload");
}

gi_status read_params(gi_nrc_s *s, float *table, float *w1, float *w2, float *w3, bool grads) {
    gi_status st = cuda_status(cudaDeviceSynchronize(), "gi_nrc parameter download");
    if (st == GI_OK && table) st = table_field(s, reinterpret_cast<float2 *>(table), grads, 0);
    const float *src = grads ? s->wg : s->w;
    cudaError_t e = cudaSuccess;
    if (st == GI_OK && w1) e = cudaMemcpy(w1, src + kW1, sizeof(float) * kHid * kIn, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && st == GI_OK && w2) e = cudaMemcpy(w2, src + kW2, sizeof(float) * kHid * kHid, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && st == GI_OK && w3) e = cudaMemcpy(w3, src + kW3, sizeof(float) * kOut * kHid, cudaMemcpyDeviceToHost);
    return st != GI_OK ? st : cuda_status(e, "gi_nrc parameter download");
}

// refresh the float16 table copy and the bf16 weight images from the masters (no Adam step)
gi_status refresh_copies(gi_nrc_s *s) {
    AdamArgs a{0.f, 0.f, 0.f, 1.f, 1.f, 1.f};
    const uint64_t entries = (uint64_t)kL * s->T;
    k_nrc_table_f16<<<(unsigned)std::min<uint64_t>((entries + 255) / 256, 65535), 256>>>(s->tab, s->tab16, entries);
    k_nrc_adam_mlp<<<(kWCount + 255) / 256, 256>>>(s->w, s->wm, s->wv, s->wg, s->wimg, 0, a);
    gi_status st = cuda_status(cudaGetLastError(), "gi_nrc copy refresh");
    if (st == GI_OK) st = cuda_status(cudaDeviceSynchronize(), "gi_nrc copy refresh");
    return st;
}

}  // namespace

namespace gi {
void nrc_route_inputs(gi_nrc_t nrc, const float **stats, float *trust, bool *trained) {
    *stats = nrc->stats;
    *trust = nrc->cfg.trust;
    *trained = nrc->steps > 0;
}

gi_status nrc_override(gi_nrc_t nrc, uint64_t n, const uint32_t **bits, const float4 **ovr) {
    if (!nrc->queried || nrc->last_query_n != n) {
        set_error("gi_probes_integrate_nrc: no gi_nrc_query_frame for a view of %llu records", (unsigned long long)n);
        return GI_ERR_INVALID_ARG;
    }
    *bits = nrc->bits;
    *ovr = nrc->ovr;
    return GI_OK;
}
}  // namespace gi

extern "C" {

gi_status gi_nrc_config_defaults(gi_nrc_config *cfg) {
    if (!cfg) {
        set_error("gi_nrc_config_defaults: NULL config");
        return GI_ERR_INVALID_ARG;
    }
    memset(cfg, 0, sizeof *cfg);
    cfg->log2_table = 19;
    // geometric level schedule from 16 to 2048 cells per axis (Mueller et al. 2022, Section 3)
    const double n_min = 16.0, n_max = 2048.0;
    const double b = pow(n_max / n_min, 1.0 / (GI_NRC_LEVELS - 1));
    for (int l = 0; l < GI_NRC_LEVELS; ++l) cfg->resolution[l] = (uint32_t)floor(n_min * pow(b, (double)l) + 1e-9);
    cfg->resolution[GI_NRC_LEVELS - 1] = (uint32_t)n_max;
    for (int a = 0; a < 3; ++a) {
        cfg->aabb_lo[a] = 0.0f;
        cfg->aabb_hi[a] = 1.0f;
    }
    cfg->lr = 1e-2f;
    cfg->beta1 = 0.9f;
    cfg->beta2 = 0.99f;
    cfg->adam_eps = 1e-15f;
    cfg->loss_eps = 0.01f;
    cfg->batch = 65536;
    cfg->train_steps = 4;
    cfg->max_records = 1u << 22;
    cfg->max_queries = 1u << 20;
    cfg->trust = 0.05f;
    cfg->query_lod = 2;
    cfg->seed = 1;
    return GI_OK;
}

gi_status gi_nrc_create(const gi_nrc_config *cfg, gi_nrc_t *out) {
    if (!cfg || !out) {
        set_error("gi_nrc_create: NULL argument");
        return GI_ERR_INVALID_ARG;
    }
    *out = nullptr;
    bool ok = cfg->log2_table >= 10 && cfg->log2_table <= 24 && cfg->lr > 0.f && cfg->beta1 >= 0.f &&
              cfg->beta1 < 1.f && cfg->beta2 >= 0.f && cfg->beta2 < 1.f && cfg->adam_eps >= 0.f &&
              cfg->loss_eps > 0.f && cfg->batch >= 128 && cfg->batch <= GI_NRC_MAX_BATCH && cfg->train_steps >= 1 &&
              cfg->batch % cfg->train_steps == 0 && cfg->batch / cfg->train_steps >= 128 && cfg->trust >= 0.f &&
              cfg->max_queries <= GI_NRC_MAX_BATCH;
    for (int l = 0; l < kL; ++l) ok = ok && cfg->resolution[l] >= 1 && cfg->resolution[l] <= (1u << 20);
    for (int a = 0; a < 3; ++a) ok = ok && std::isfinite(cfg->aabb_lo[a]) && std::isfinite(cfg->aabb_hi[a]) &&
                                     cfg->aabb_hi[a] > cfg->aabb_lo[a];
    if (!ok) {
        set_error("gi_nrc_create: configuration out of range");
        return GI_ERR_INVALID_ARG;
    }
    gi_nrc_s *s = new gi_nrc_s();
    s->cfg = *cfg;
    s->T = 1u << cfg->log2_table;
    s->sms = sm_count();
    for (int a = 0; a < 3; ++a) {
        s->geo.lo[a] = cfg->aabb_lo[a];
        s->geo.inv_ext[a] = (float)(1.0 / ((double)cfg->aabb_hi[a] - (double)cfg->aabb_lo[a]));
    }
    s->geo.log2_table = cfg->log2_table;
    for (int l = 0; l < kL; ++l) {
        const uint64_t V = (uint64_t)cfg->resolution[l] + 1u;
        s->geo.lv.res[l] = cfg->resolution[l];
        s->geo.lv.dense[l] = 6u * V * V * V <= s->T ? 1u : 0u;
    }
    const size_t entries = (size_t)kL * s->T;
    gi_status st = nrc_alloc((void **)&s->tab, entries * sizeof(Entry));
    if (st == GI_OK) st = nrc_alloc((void **)&s->grad, entries * sizeof(float2));
    if (st == GI_OK) st = nrc_alloc((void **)&s->tab16, entries * sizeof(__half2));
    if (st == GI_OK) st = nrc_alloc((void **)&s->w, kWCount * 4);
    if (st == GI_OK) st = nrc_alloc((void **)&s->wm, kWCount * 4);
    if (st == GI_OK) st = nrc_alloc((void **)&s->wv, kWCount * 4);
    if (st == GI_OK) st = nrc_alloc((void **)&s->wg, kWCount * 4);
    if (st == GI_OK) st = nrc_alloc((void **)&s->wimg, kImgBytes);
    if (st == GI_OK) st = nrc_alloc((void **)&s->stats, 16);
    if (st == GI_OK) st = nrc_alloc((void **)&s->wpart, (size_t)s->sms * kPartStride * 4);
    if (st == GI_OK) st = nrc_alloc((void **)&s->err, 4);
    if (st == GI_OK) st = nrc_alloc((void **)&s->qcount, 4);
    const uint32_t maxr = std::max<uint32_t>(cfg->max_records, 32);
    if (st == GI_OK) st = nrc_alloc((void **)&s->bits, ((size_t)maxr + 31) / 32 * 4 + 8);
    if (st == GI_OK) st = nrc_alloc((void **)&s->ovr, (size_t)maxr * sizeof(float4));
    if (st == GI_OK) st = nrc_alloc((void **)&s->qidx, (size_t)std::max<uint32_t>(cfg->max_queries, 1) * 4);
    if (st == GI_OK) st = ensure_capacity(s, std::max(cfg->batch, cfg->max_queries));
    if (st != GI_OK) {
        nrc_free(s);
        delete s;
        return st;
    }
    cudaError_t e = cudaMemset(s->tab, 0, entries * sizeof(Entry));
    if (e == cudaSuccess) e = cudaMemset(s->grad, 0, entries * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemset(s->wm, 0, kWCount * 4);
    if (e == cudaSuccess) e = cudaMemset(s->wv, 0, kWCount * 4);
    if (e == cudaSuccess) e = cudaMemset(s->wg, 0, kWCount * 4);
    if (e == cudaSuccess) e = cudaMemset(s->wimg, 0, kImgBytes);
    if (e == cudaSuccess) e = cudaMemset(s->stats, 0, 16);
    if (e == cudaSuccess) e = cudaMemset(s->err, 0, 4);
    if (e == cudaSuccess) e = cudaMemset(s->qcount, 0, 4);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_nrc_mlp<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmTrain);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_nrc_mlp<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmInfer);
    st = cuda_status(e, "gi_nrc_create");
    if (st == GI_OK) {
        // initial parameters from a splitmix64 stream: table, then W1, W2, W3
        uint64_t rs = cfg->seed;
        std::vector<float> table(entries * 2);
        for (auto &v : table) v = (float)(uniform01(rs) * 2e-4 - 1e-4);
        std::vector<float> w(kWCount);
        const double b1 = std::sqrt(6.0 / (kIn + kHid)), b2 = std::sqrt(6.0 / (kHid + kHid)),
                     b3 = std::sqrt(6.0 / (kHid + kOut));
        for (int i = 0; i < kWCount; ++i) {
            const double b = i < kW2 ? b1 : (i < kW3 ? b2 : b3);
            w[i] = (float)((uniform01(rs) * 2.0 - 1.0) * b);
        }
        st = copy_params(s, table.data(), w.data() + kW1, w.data() + kW2, w.data() + kW3, false);
        if (st == GI_OK) st = refresh_copies(s);
    }
    if (st != GI_OK) {
        nrc_free(s);
        delete s;
        return st;
    }
    *out = s;
    return GI_OK;
}

gi_status gi_nrc_destroy(gi_nrc_t nrc) {
    if (!nrc) return GI_OK;
    cudaDeviceSynchronize();
    nrc_free(nrc);
    delete nrc;
    return GI_OK;
}

gi_status gi_nrc_set_params(gi_nrc_t nrc, const float *table, const float *w1, const float *w2, const float *w3) {
    if (!nrc) {
        set_error("gi_nrc_set_params: NULL surrogate");
        return GI_ERR_INVALID_ARG;
    }
    gi_status st = cuda_status(cudaDeviceSynchronize(), "gi_nrc_set_params");
    if (st != GI_OK) return st;
    // reset Adam moments and gradients (the whole entry but the master features)
    st = table_field(nrc, nullptr, false, 2);
    if (st != GI_OK) return st;
    cudaError_t e = cudaMemset(nrc->grad, 0, (size_t)kL * nrc->T * sizeof(float2));
    if (e == cudaSuccess) e = cudaMemset(nrc->wm, 0, kWCount * 4);
    if (e == cudaSuccess) e = cudaMemset(nrc->wv, 0, kWCount * 4);
    if (e == cudaSuccess) e = cudaMemset(nrc->wg, 0, kWCount * 4);
    st = cuda_status(e, "gi_nrc_set_params");
    if (st == GI_OK) st = copy_params(nrc, table, w1, w2, w3, false);
    if (st == GI_OK) st = refresh_copies(nrc);
    nrc->steps = 0;
    return st;
}

gi_status gi_nrc_get_params(gi_nrc_t nrc, float *table, float *w1, float *w2, float *w3) {
    if (!nrc) {
        set_error("gi_nrc_get_params: NULL surrogate");
        return GI_ERR_INVALID_ARG;
    }
    return read_params(nrc, table, w1, w2, w3, false);
}

gi_status gi_nrc_set_gradients(gi_nrc_t nrc, const float *table, const float *w1, const float *w2, const float *w3) {
    if (!nrc) {
        set_error("gi_nrc_set_gradients: NULL surrogate");
        return GI_ERR_INVALID_ARG;
    }
    gi_status st = cuda_status(cudaDeviceSynchronize(), "gi_nrc_set_gradients");
    if (st == GI_OK) st = copy_params(nrc, table, w1, w2, w3, true);
    return st;
}

gi_status gi_nrc_get_gradients(gi_nrc_t nrc, float *table, float *w1, float *w2, float *w3) {
    if (!nrc) {
        set_error("gi_nrc_get_gradients: NULL surrogate");
        return GI_ERR_INVALID_ARG;
    }
    return read_params(nrc, table, w1, w2, w3, true);
}

gi_status gi_nrc_infer(gi_nrc_t nrc, const gi_points *pts, float *out, gi_stream_t stream) {
    if (!nrc || !points_ok(pts) || (!out && pts->n)) {
        set_error("gi_nrc_infer: NULL argument or more than GI_NRC_MAX_BATCH points");
        return GI_ERR_INVALID_ARG;
    }
    if (pts->n == 0) return GI_OK;
    gi_status st = ensure_capacity(nrc, pts->n);
    if (st != GI_OK) return st;
    const cudaStream_t s = (cudaStream_t)stream;
    EncArgs e = enc_base(nrc);
    for (int a = 0; a < 3; ++a) {
        e.pos[a] = pts->pos[a];
        e.nrm[a] = pts->nrm[a];
    }
    e.n = pts->n;
    e.T = nullptr;
    const uint32_t n_pad = (pts->n + kTile - 1) / kTile * kTile;
    k_nrc_encode<kEncPoints><<<enc_blocks(nrc, (uint64_t)n_pad * kL), kEncThreads, 0, s>>>(e);
    st = cuda_status(cudaGetLastError(), "k_nrc_encode launch");
    if (st == GI_OK) st = launch_mlp(nrc, false, pts->n, nullptr, 0.f, reinterpret_cast<float4 *>(out), nullptr, s);
    return st;
}

gi_status gi_nrc_backward(gi_nrc_t nrc, const gi_points *pts, const float *const target[3], const float *mask,
                          uint32_t batch_norm, gi_stream_t stream) {
    if (!nrc || !points_ok(pts) || !target || (pts->n && (!target[0] || !target[1] || !target[2]))) {
        set_error("gi_nrc_backward: NULL argument or more than GI_NRC_MAX_BATCH points");
        return GI_ERR_INVALID_ARG;
    }
    const cudaStream_t s = (cudaStream_t)stream;
    gi_status st = cuda_status(cudaMemsetAsync(nrc->stats, 0, 16, s), "gi_nrc_backward");
    if (st != GI_OK || pts->n == 0) return st;
    st = ensure_capacity(nrc, pts->n);
    if (st != GI_OK) return st;
    EncArgs e = enc_base(nrc);
    for (int a = 0; a < 3; ++a) {
        e.pos[a] = pts->pos[a];
        e.nrm[a] = pts->nrm[a];
        e.target[a] = target[a];
    }
    e.mask = mask;
    e.n = pts->n;
    const uint32_t n_pad = (pts->n + kTile - 1) / kTile * kTile;
    k_nrc_encode<kEncPoints><<<enc_blocks(nrc, (uint64_t)n_pad * kL), kEncThreads, 0, s>>>(e);
    st = cuda_status(cudaGetLastError(), "k_nrc_encode launch");
    const float B = (float)(batch_norm ? batch_norm : pts->n);
    nrc->last_minibatches = 1;
    if (st == GI_OK) st = launch_mlp(nrc, true, pts->n, nullptr, 2.0f / B, nullptr, nullptr, s);
    if (st == GI_OK) st = scatter_and_return(nrc, pts->pos, pts->nrm, nullptr, pts->n, s);
    return st;
}

gi_status gi_nrc_set_learning_rate(gi_nrc_t nrc, float lr) {
    if (!nrc || !(lr > 0.0f) || !std::isfinite(lr)) {
        set_error("gi_nrc_set_learning_rate: NULL surrogate or step size not finite and > 0");
        return GI_ERR_INVALID_ARG;
    }
    nrc->cfg.lr = lr;
    return GI_OK;
}

gi_status gi_nrc_adam(gi_nrc_t nrc, gi_stream_t stream) {
    if (!nrc) {
        set_error("gi_nrc_adam: NULL surrogate");
        return GI_ERR_INVALID_ARG;
    }
    const cudaStream_t s = (cudaStream_t)stream;
    nrc->steps += 1;
    const double t = (double)nrc->steps;
    AdamArgs a;
    a.lr = nrc->cfg.lr;
    a.b1 = nrc->cfg.beta1;
    a.b2 = nrc->cfg.beta2;
    a.eps = nrc->cfg.adam_eps;
    a.c1 = (float)(1.0 - std::pow((double)nrc->cfg.beta1, t));
    a.c2 = (float)(1.0 - std::pow((double)nrc->cfg.beta2, t));
    const uint64_t entries = (uint64_t)kL * nrc->T;
    const unsigned blocks = (unsigned)std::min<uint64_t>((entries / 4 + 255) / 256, (uint64_t)nrc->sms * 8);
    k_nrc_adam_table<<<blocks, 256, 0, s>>>(nrc->tab, nrc->grad, nrc->tab16, entries, a);
    gi_status st = cuda_status(cudaGetLastError(), "k_nrc_adam_table launch");
    if (st != GI_OK) return st;
    k_nrc_adam_mlp<<<(kWCount + 255) / 256, 256, 0, s>>>(nrc->w, nrc->wm, nrc->wv, nrc->wg, nrc->wimg, 1, a);
    return cuda_status(cudaGetLastError(), "k_nrc_adam_mlp launch");
}

gi_status gi_nrc_train_frame(gi_nrc_t nrc, gi_cache_t cache, const gi_hits *hits, const uint32_t *slot_ids,
                             uint32_t frame, gi_stream_t stream) {
    if (!nrc || !cache || !hits || !slot_ids || !hits->ray_len || hits->n == 0 || hits->n > nrc->cfg.max_records ||
        hits->n > 0xFFFFFFFFull) {
        set_error("gi_nrc_train_frame: NULL argument, no records, or more than max_records");
        return GI_ERR_INVALID_ARG;
    }
    for (int a = 0; a < 3; ++a)
        if (!hits->pos[a] || !hits->nrm[a]) {
            set_error("gi_nrc_train_frame: NULL record plane");
            return GI_ERR_INVALID_ARG;
        }
    const cudaStream_t s = (cudaStream_t)stream;
    gi_status st = cuda_status(cudaMemsetAsync(nrc->stats, 0, 16, s), "gi_nrc_train_frame");
    if (st != GI_OK) return st;
    const uint32_t steps = nrc->cfg.train_steps, B = nrc->cfg.batch / steps;
    EncArgs e = enc_base(nrc);
    for (int a = 0; a < 3; ++a) {
        e.pos[a] = hits->pos[a];
        e.nrm[a] = hits->nrm[a];
    }
    e.len = hits->ray_len;
    e.n = B;
    e.n_records = (uint32_t)hits->n;
    e.seed = pcg_hash(frame + 1u);
    e.slot_ids = slot_ids;
    e.cv = cache_view(cache);
    const uint32_t n_pad = (B + kTile - 1) / kTile * kTile;
    for (uint32_t j = 0; j < steps && st == GI_OK; ++j) {
        e.offset = j * B;
        k_nrc_encode<kEncSampled><<<enc_blocks(nrc, (uint64_t)n_pad * kL), kEncThreads, 0, s>>>(e);
        st = cuda_status(cudaGetLastError(), "k_nrc_encode launch");
        if (st == GI_OK) st = launch_mlp(nrc, true, B, nullptr, 2.0f / (float)B, nullptr, nullptr, s);
        if (st == GI_OK) st = scatter_and_return(nrc, hits->pos, hits->nrm, nrc->idx, B, s);
        if (st == GI_OK) st = gi_nrc_adam(nrc, stream);
    }
    nrc->last_minibatches = steps;
    return st;
}

gi_status gi_nrc_query_frame(gi_nrc_t nrc, gi_cache_t cache, const gi_hits *hits, const uint32_t *slot_ids,
                             const gi_view *view, gi_stream_t stream) {
    if (!nrc || !cache || !hits || !slot_ids || !hits->ray_len || !view_ok(view) || hits->n > nrc->cfg.max_records) {
        set_error("gi_nrc_query_frame: NULL argument, bad view, or more than max_records");
        return GI_ERR_INVALID_ARG;
    }
    for (int a = 0; a < 3; ++a)
        if (!hits->pos[a] || !hits->nrm[a]) {
            set_error("gi_nrc_query_frame: NULL record plane");
            return GI_ERR_INVALID_ARG;
        }
    const cudaStream_t s = (cudaStream_t)stream;
    gi_status st = cuda_status(cudaMemsetAsync(nrc->qcount, 0, 4, s), "gi_nrc_query_frame");
    if (st != GI_OK) return st;
    nrc->queried = true;
    nrc->last_query_n = hits->n;
    if (hits->n == 0) return GI_OK;
    SelectArgs a;
    for (int k = 0; k < 3; ++k) a.pos[k] = hits->pos[k];
    a.len = hits->ray_len;
    a.slot_ids = slot_ids;
    a.n = (uint32_t)hits->n;
    a.cv = cache_view(cache);
    a.kp = cache_update_args(cache, hits, view, nullptr).kp;
    a.query_lod = nrc->cfg.query_lod;
    a.trust = nrc->cfg.trust;
    a.trained = nrc->steps > 0 ? 1u : 0u;
    a.stats = nrc->stats;
    a.max_q = nrc->cfg.max_queries;
    a.qidx = nrc->qidx;
    a.qcount = nrc->qcount;
    a.bits = nrc->bits;
    const uint32_t words = (a.n + 31u) / 32u;
    const unsigned blocks = (unsigned)std::max<uint32_t>(1, std::min<uint32_t>((words + 7) / 8, (uint32_t)nrc->sms * 8));
    k_nrc_select<<<blocks, 256, 0, s>>>(a);
    st = cuda_status(cudaGetLastError(), "k_nrc_select launch");
    if (st != GI_OK || nrc->cfg.max_queries == 0) return st;
    EncArgs e = enc_base(nrc);
    for (int k = 0; k < 3; ++k) {
        e.pos[k] = hits->pos[k];
        e.nrm[k] = hits->nrm[k];
    }
    e.len = hits->ray_len;
    e.n = nrc->cfg.max_queries;
    e.qidx = nrc->qidx;
    e.qcount = nrc->qcount;
    e.T = nullptr;
    k_nrc_encode<kEncQueries><<<(unsigned)nrc->sms * 8, kEncThreads, 0, s>>>(e);
    st = cuda_status(cudaGetLastError(), "k_nrc_encode launch");
    if (st == GI_OK) st = launch_mlp(nrc, false, nrc->cfg.max_queries, nrc->qcount, 0.f, nrc->ovr, nrc->qidx, s);
    return st;
}

gi_status gi_nrc_answers(gi_nrc_t nrc, uint32_t *records, float *rad, uint32_t capacity, uint32_t *count,
                         gi_stream_t stream) {
    if (!nrc || !count || (capacity && (!records || !rad))) {
        set_error("gi_nrc_answers: NULL argument");
        return GI_ERR_INVALID_ARG;
    }
    const cudaStream_t s = (cudaStream_t)stream;
    uint32_t c = 0;
    gi_status st = cuda_status(cudaStreamSynchronize(s), "gi_nrc_answers");
    if (st == GI_OK) st = cuda_status(cudaMemcpy(&c, nrc->qcount, 4, cudaMemcpyDeviceToHost), "gi_nrc_answers");
    if (st != GI_OK) return st;
    c = std::min(c, nrc->cfg.max_queries);
    *count = c;
    if (capacity == 0 && !records) return GI_OK;
    if (c > capacity) {
        set_error("gi_nrc_answers: %u answers, capacity %u", c, capacity);
        return GI_ERR_CAPACITY;
    }
    if (c) {
        k_nrc_gather_answers<<<(c + 255) / 256, 256, 0, s>>>(nrc->qidx, nrc->ovr, c, records,
                                                               reinterpret_cast<float4 *>(rad));
        st = cuda_status(cudaGetLastError(), "k_nrc_gather_answers launch");
        if (st == GI_OK) st = cuda_status(cudaStreamSynchronize(s), "gi_nrc_answers");
    }
    return st;
}

gi_status gi_nrc_stats(gi_nrc_t nrc, gi_nrc_stats_t *out, gi_stream_t stream) {
    if (!nrc || !out) {
        set_error("gi_nrc_stats: NULL argument");
        return GI_ERR_INVALID_ARG;
    }
    float st4[4];
    uint32_t q = 0, err = 0;
    gi_status st = cuda_status(cudaStreamSynchronize((cudaStream_t)stream), "gi_nrc_stats");
    if (st == GI_OK) st = cuda_status(cudaMemcpy(st4, nrc->stats, 16, cudaMemcpyDeviceToHost), "gi_nrc_stats");
    if (st == GI_OK) st = cuda_status(cudaMemcpy(&q, nrc->qcount, 4, cudaMemcpyDeviceToHost), "gi_nrc_stats");
    if (st == GI_OK) st = cuda_status(cudaMemcpy(&err, nrc->err, 4, cudaMemcpyDeviceToHost), "gi_nrc_stats");
    if (st != GI_OK) return st;
    out->steps = nrc->steps;
    out->loss = st4[0] / (float)nrc->last_minibatches;
    out->judged_error = st4[2] > 0.f ? st4[1] / st4[2] : 0.f;
    out->trusted = (nrc->steps > 0 && st4[2] > 0.f && st4[1] <= nrc->cfg.trust * st4[2]) ? 1u : 0u;
    out->queries = nrc->queried ? std::min(q, nrc->cfg.max_queries) : 0u;
    if (err) {
        set_error("gi_nrc: a bounded tensor-core wait ran out (error word %u)", err);
        return GI_ERR_TIMEOUT;
    }
    return GI_OK;
}

}  // extern "C"
