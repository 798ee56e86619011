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

// Cache internals needed by the probe kernels.
struct CacheView {
    const void *resolved;      // resolved radiance of slot 0: float4, or half4 (ushort4)
    uint32_t resolved_stride;  // bytes between the resolved values of consecutive slots
    int resolved_f16;
    uint32_t slots;
};
CacheView cache_view(gi_cache_t c);

} // namespace gi

// ---------------------------------------------------------------- device helpers
namespace gi {

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
