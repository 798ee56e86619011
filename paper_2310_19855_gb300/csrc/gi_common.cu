// Error reporting and per-view constants shared by the cache and probe passes.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "gi_internal.cuh"

namespace gi {

static thread_local char g_err[512] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
}

gi_status cuda_status(cudaError_t e, const char *what) {
    if (e == cudaSuccess) return GI_OK;
    set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    if (e == cudaErrorMemoryAllocation) return GI_ERR_OOM;
    return GI_ERR_CUDA;
}

// Algorithm 6: cell_size(d) = tan(fov_y * proj_size * max(1/H, H/W^2)) * d, proj_size = 8.
double distance_scale(double fov_y, uint32_t width, uint32_t height) {
    double w = (double)width, h = (double)height;
    double m = fmax(1.0 / h, h / (w * w));
    return tan(fov_y * 8.0 * m);
}

bool view_ok(const gi_view *v) {
    if (!v) return false;
    if (v->width == 0 || v->height == 0 || v->width > 65535 || v->height > 65535) return false;
    if (!(v->fov_y > 0.0 && v->fov_y < 3.14)) return false;
    return true;
}

// LOD l has side s0 2^l; it is chosen where d^2 >= T_(l-1), T_k = (2^(k+1) s0 / distance_scale)^2,
// i.e. where Algorithm 6's cell size reaches s0 2^l.  Everything is evaluated in double and
// rounded to float once; 1/s_l is the float of 1/s0 scaled by 2^-l (exact).
KeyParams key_params(float cell_size, uint32_t num_lods, const gi_view *v) {
    KeyParams k;
    double s0 = (double)cell_size;
    double ds = distance_scale(v->fov_y, v->width, v->height);
    double d0 = s0 / ds;
    for (int i = 0; i < 3; ++i) {
        double r = d0 * ldexp(1.0, i + 1);
        k.thr[i] = (float)(r * r);
    }
    float inv0 = (float)(1.0 / s0);
    for (int l = 0; l < 4; ++l) {
        k.side[l] = (float)(s0 * ldexp(1.0, l));
        k.inv_side[l] = (float)((double)inv0 * ldexp(1.0, -l));
    }
    for (int a = 0; a < 3; ++a) k.cam[a] = v->cam_pos[a];
    k.num_lods = (int)num_lods;
    return k;
}

CamParams cam_params(const gi_view *v) {
    CamParams c;
    for (int a = 0; a < 3; ++a) {
        c.pos[a] = v->cam_pos[a];
        c.fwd[a] = v->cam_fwd[a];
        c.right[a] = v->cam_right[a];
        c.up[a] = v->cam_up[a];
    }
    double th = tan(0.5 * v->fov_y);
    c.sy_scale = (float)th;
    c.sx_scale = (float)(th * (double)v->width / (double)v->height);
    c.inv_w = (float)(1.0 / (double)v->width);
    c.inv_h = (float)(1.0 / (double)v->height);
    c.width = v->width;
    c.height = v->height;
    return c;
}

} // namespace gi

extern "C" {

const char *gi_last_error(void) { return gi::g_err; }

const char *gi_status_string(gi_status s) {
    switch (s) {
    case GI_OK: return "GI_OK";
    case GI_ERR_INVALID_ARG: return "GI_ERR_INVALID_ARG";
    case GI_ERR_OOM: return "GI_ERR_OOM";
    case GI_ERR_CUDA: return "GI_ERR_CUDA";
    case GI_ERR_TIMEOUT: return "GI_ERR_TIMEOUT";
    case GI_ERR_DEVICE_FAULT: return "GI_ERR_DEVICE_FAULT";
    case GI_ERR_CAPACITY: return "GI_ERR_CAPACITY";
    case GI_WARN_DROPPED: return "GI_WARN_DROPPED";
    }
    return "GI_UNKNOWN";
}

uint32_t gi_version(void) { return 100; }

} // extern "C"
