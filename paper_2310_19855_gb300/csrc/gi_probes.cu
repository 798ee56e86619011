// Screen probes (Section 2.1): spawn per 8x8 tile with a Halton jitter
// (2.1.1), probe mask + MIP chain and the directional search of Algorithm 3
// (2.1.5), probe irradiance through 3-band spherical harmonics (2.1.4, 2.4.2)
// and per-pixel interpolation (2.4.1).
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include <mutex>

#include "gi_internal.cuh"

namespace gi {

constexpr unsigned kFullMask = 0xFFFFFFFFu;


static MipInfo mip_info(const gi_probe_layout &l) {
    MipInfo m;
    memset(&m, 0, sizeof m);
    m.count = (int)l.mip_count;
    for (int k = 0; k < (int)l.mip_count; ++k) {
        m.w[k] = (int)l.mip_w[k];
        m.h[k] = (int)l.mip_h[k];
        m.off[k] = (int)l.mip_offset[k];
    }
    return m;
}

// ---------------------------------------------------------------- cell moments
// Per hemi-octahedral cell (local frame): solid angle, first moment, second
// moment (xx yy zz xy xz yz).  Table layout [moment][cell] for coalesced reads.
__device__ float g_moments[10][64];

// Each cell is a spherical quadrilateral: the octahedral map sends the straight
// sides of the (u, v) square to straight segments, i.e. great-circle arcs.
// Closed forms on a spherical polygon with counter-clockwise vertices a_k:
//   solid angle   -- sum of triangle-fan excesses (Van Oosterom & Strackee 1983)
//   first moment  -- 1/2 sum_k theta_k n_k  (Arvo 1995), n_k = unit(a_k x a_k+1)
//   second moment -- 1/3 (Omega I + sum_k e_k n_k^T), e_k = integral of the
//                    direction along arc k = a sin(theta) + c (1 - cos(theta)),
//                    c the in-plane unit vector orthogonal to a towards b
//                    (Stokes' theorem on the sphere applied to w_i w).
static void hemioct_dir(double u, double v, double out[3]) {
    double x = 0.5 * (u + v), y = 0.5 * (u - v);
    double z = 1.0 - fabs(x) - fabs(y);
    double n = sqrt(x * x + y * y + z * z);
    out[0] = x / n;
    out[1] = y / n;
    out[2] = z / n;
}

static void cross3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static void cell_moments_closed_form(int c, double out[10]) {
    const double h = 0.25;
    const double u0 = -1.0 + (c & 7) * h, v0 = -1.0 + (c >> 3) * h;
    // (u, v) -> (x, y) has determinant -1/2: reverse the square's order to get
    // counter-clockwise seen from outside the sphere.
    double V[4][3];
    hemioct_dir(u0, v0, V[0]);
    hemioct_dir(u0, v0 + h, V[1]);
    hemioct_dir(u0 + h, v0 + h, V[2]);
    hemioct_dir(u0 + h, v0, V[3]);
    double omega = 0.0;
    for (int k = 1; k < 3; ++k) {
        double bc[3];
        cross3(V[k], V[k + 1], bc);
        double num = dot3(V[0], bc);
        double den = 1.0 + dot3(V[0], V[k]) + dot3(V[k], V[k + 1]) + dot3(V[k + 1], V[0]);
        omega += 2.0 * atan2(num, den);
    }
    double m1[3] = {0, 0, 0};
    double m2[3][3] = {{omega, 0, 0}, {0, omega, 0}, {0, 0, omega}};
    for (int k = 0; k < 4; ++k) {
        const double *a = V[k], *b = V[(k + 1) & 3];
        double cr[3];
        cross3(a, b, cr);
        double sn = sqrt(dot3(cr, cr));
        double cs = dot3(a, b);
        double th = atan2(sn, cs);
        double nk[3] = {cr[0] / sn, cr[1] / sn, cr[2] / sn};
        double e[3];
        for (int i = 0; i < 3; ++i) {
            double cdir = (b[i] - a[i] * cs) / sn;
            e[i] = a[i] * sn + cdir * (1.0 - cs);
            m1[i] += 0.5 * th * nk[i];
        }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) m2[i][j] += e[i] * nk[j];
    }
    out[0] = omega;
    for (int i = 0; i < 3; ++i) out[1 + i] = m1[i];
    const double s = 1.0 / 3.0;
    out[4] = s * m2[0][0];
    out[5] = s * m2[1][1];
    out[6] = s * m2[2][2];
    out[7] = s * 0.5 * (m2[0][1] + m2[1][0]);
    out[8] = s * 0.5 * (m2[0][2] + m2[2][0]);
    out[9] = s * 0.5 * (m2[1][2] + m2[2][1]);
}

// Local unit direction of each cell's centre (u, v) = (-1 + (i + 1/2)/4, -1 + (j + 1/2)/4), cell 8 j + i.
// In global memory (read through the read-only cache): the filter reads it at a different index in
// every lane, which the constant cache would serialise.
__device__ float g_cell_dir[64][3];
// cos(pi / 50): the angle-error threshold of the probe filter (Algorithm 5)
__constant__ float c_filter_cos;

static std::mutex g_moments_mutex;
static bool g_moments_ready[64];

gi_status ensure_moments() {
    int dev = 0;
    gi_status s = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
    if (s != GI_OK) return s;
    std::lock_guard<std::mutex> lock(g_moments_mutex);
    if (dev >= 0 && dev < 64 && g_moments_ready[dev]) return GI_OK;
    float table[10][64];
    for (int c = 0; c < 64; ++c) {
        double m[10];
        cell_moments_closed_form(c, m);
        for (int k = 0; k < 10; ++k) table[k][c] = (float)m[k];
    }
    s = cuda_status(cudaMemcpyToSymbol(g_moments, table, sizeof table), "upload cell moments");

    float dirs[64][3];
    for (int c = 0; c < 64; ++c) {
        const double u = -1.0 + ((c & 7) + 0.5) * 0.25, v = -1.0 + ((c >> 3) + 0.5) * 0.25;
        const double x = 0.5 * (u + v), y = 0.5 * (u - v), z = 1.0 - fabs(x) - fabs(y);
        const double n = sqrt(x * x + y * y + z * z);
        dirs[c][0] = (float)(x / n);
        dirs[c][1] = (float)(y / n);
        dirs[c][2] = (float)(z / n);
    }
    const float fc = (float)cos(3.14159265358979323846 / 50.0);
    if (s == GI_OK) s = cuda_status(cudaMemcpyToSymbol(g_cell_dir, dirs, sizeof dirs), "upload cell directions");
    if (s == GI_OK) s = cuda_status(cudaMemcpyToSymbol(c_filter_cos, &fc, sizeof fc), "upload filter threshold");
    if (s == GI_OK && dev >= 0 && dev < 64) g_moments_ready[dev] = true;
    return s;
}

// ---------------------------------------------------------------- spawn

// Block of 16x16 tiles: level 0 plus levels 1..4 of its region, built in shared memory.  With
// temporal upscale u, the 8x8 tile holding the probe pixel min(8u S + jitter, image) of its spawn
// tile S = tile / u receives the fresh probe (Section 2.1.1); with keep, the other tiles (and a
// fresh tile whose pixel is sky) keep what level 0 holds (the reprojected probes).
__device__ __forceinline__ void spawn_body(const SpawnArgs &a, uint32_t bx, uint32_t by) {
    __shared__ uint32_t s_lvl[2][16][16];
    const int lx = threadIdx.x & 15, ly = threadIdx.x >> 4;
    const uint32_t tx = bx * 16 + lx, ty = by * 16 + ly;
    uint32_t m = GI_PROBE_NONE;
    if (tx < a.tiles_x && ty < a.tiles_y) {
        const uint32_t st = 8u * a.upscale;
        const uint32_t px = min(st * (tx / a.upscale) + (uint32_t)a.jx, a.width - 1u);
        const uint32_t py = min(st * (ty / a.upscale) + (uint32_t)a.jy, a.height - 1u);
        const uint32_t p = ty * a.tiles_x + tx;
        bool fresh = false;
        float4 nd = make_float4(0.f, 0.f, 0.f, 0.f);
        if ((px >> 3) == tx && (py >> 3) == ty) {
            nd = __ldg(a.gbuf + (size_t)py * a.width + px);
            fresh = isfinite(nd.w) && nd.w >= 0.0f;
        }
        if (fresh) {
            m = (py << 16) | px;
            const float3 w = pixel_world_exact(a.cam, px, py, nd.w);
            a.pos[p] = make_float4(w.x, w.y, w.z, nd.w);
            a.nrm[p] = make_float4(nd.x, nd.y, nd.z, 1.0f);
            a.mask[p] = m;
        } else if (a.keep) {
            m = a.mask[p];
        } else {
            a.pos[p] = make_float4(0.f, 0.f, 0.f, 0.f);
            a.nrm[p] = make_float4(0.f, 0.f, 0.f, 0.f);
            a.mask[p] = m;
        }
    }
    s_lvl[0][ly][lx] = m;
    __syncthreads();
    // level L keeps the first valid probe of each 2x2 block in the order (0,0), (1,0), (0,1), (1,1)
    for (int L = 1; L <= 4 && L < a.mi.count; ++L) {
        const int n = 16 >> L;
        const int src = (L - 1) & 1, dst = L & 1;
        uint32_t v = GI_PROBE_NONE;
        const int x = threadIdx.x % n, y = threadIdx.x / n;
        if ((int)threadIdx.x < n * n) {
            const uint32_t c0 = s_lvl[src][2 * y][2 * x], c1 = s_lvl[src][2 * y][2 * x + 1];
            const uint32_t c2 = s_lvl[src][2 * y + 1][2 * x], c3 = s_lvl[src][2 * y + 1][2 * x + 1];
            v = c0 != GI_PROBE_NONE ? c0 : (c1 != GI_PROBE_NONE ? c1 : (c2 != GI_PROBE_NONE ? c2 : c3));
        }
        __syncthreads();
        if ((int)threadIdx.x < n * n) {
            s_lvl[dst][y][x] = v;
            const int X = bx * n + x, Y = by * n + y;
            if (X < a.mi.w[L] && Y < a.mi.h[L]) a.mask[a.mi.off[L] + Y * a.mi.w[L] + X] = v;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_spawn(SpawnArgs a) { spawn_body(a, blockIdx.x, blockIdx.y); }

// Levels 5 and up, from level 4, in one block.
__device__ __forceinline__ void mip_tail_body(uint32_t *mask, const MipInfo &mi) {
    for (int L = 5; L < mi.count; ++L) {
        const int w = mi.w[L], h = mi.h[L], pw = mi.w[L - 1], ph = mi.h[L - 1];
        const uint32_t *src = mask + mi.off[L - 1];
        for (int t = threadIdx.x; t < w * h; t += blockDim.x) {
            const int x = t % w, y = t / w;
            uint32_t v = GI_PROBE_NONE;
            const int cx[4] = {2 * x, 2 * x + 1, 2 * x, 2 * x + 1}, cy[4] = {2 * y, 2 * y, 2 * y + 1, 2 * y + 1};
            for (int k = 0; k < 4 && v == GI_PROBE_NONE; ++k)
                if (cx[k] < pw && cy[k] < ph) v = __ldcg(src + cy[k] * pw + cx[k]);
            mask[mi.off[L] + y * w + x] = v;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(1024) k_mip_tail(uint32_t *mask, MipInfo mi) { mip_tail_body(mask, mi); }

// ---------------------------------------------------------------- probe irradiance

__device__ __forceinline__ float3 fetch_resolved(const void *r, uint32_t stride, int f16, uint32_t s) {
    r = static_cast<const char *>(r) + (size_t)s * stride;
    if (f16) {
        const ushort4 h = __ldg(reinterpret_cast<const ushort4 *>(r));
        return make_float3(__half2float(__ushort_as_half(h.x)), __half2float(__ushort_as_half(h.y)),
                           __half2float(__ushort_as_half(h.z)));
    }
    const float4 v = __ldg(reinterpret_cast<const float4 *>(r));
    return make_float3(v.x, v.y, v.z);
}

__device__ __forceinline__ bool ray_sample(const IntegrateArgs &a, uint32_t s, float3 &r) {
    if (s < a.slots) {
        r = fetch_resolved(a.resolved, a.res_stride, a.f16, s);
        return true;
    }
    r = make_float3(a.env[0], a.env[1], a.env[2]);
    return s == GI_SLOT_MISS;
}

// Cell radiance of probe p's rays (one warp; lane l owns cells l and l + 32, ray k samples cell
// k mod 64): L = per-cell mean of the rays that produced a sample, with the radiance backup (mean
// over populated cells) where none did; with HITDIST also hd = the mean ray length of the cell's
// rays that hit a surface (+inf when none did).  With SURR, records whose bit is set in
// a.ovr_bits take their radiance from a.ovr (the surrogate's answers) instead of the cache.
template <bool SURR, bool HITDIST>
__device__ __forceinline__ void gather_cells(const IntegrateArgs &a, uint32_t p, int lane, float (&L)[2][3],
                                             float (&hd)[2]) {
    float acc[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float cnt[2] = {0.f, 0.f};
    float hs[2] = {0.f, 0.f}, hn[2] = {0.f, 0.f};
    const uint32_t *ids = a.slot_ids + (size_t)p * a.rpp;
    for (uint32_t k = lane; k < a.rpp; k += 64) {
        // rays k and k + 32 sample cells lane and lane + 32; both gathers in flight together
        const uint32_t s0 = __ldcs(ids + k), s1 = __ldcs(ids + k + 32);
        float3 r0, r1;
        bool h0 = ray_sample(a, s0, r0), h1 = ray_sample(a, s1, r1);
        if (SURR) {
            // rpp is a multiple of 64: rays k and k + 32 are bit `lane` of two consecutive words
            const size_t rec = (size_t)p * a.rpp + k;
            const uint32_t w0 = __ldg(a.ovr_bits + (rec >> 5)), w1 = __ldg(a.ovr_bits + (rec >> 5) + 1);
            if ((w0 >> lane) & 1u) {
                const float4 o = __ldg(a.ovr + rec);
                r0 = make_float3(o.x, o.y, o.z);
                h0 = true;
            }
            if ((w1 >> lane) & 1u) {
                const float4 o = __ldg(a.ovr + rec + 32);
                r1 = make_float3(o.x, o.y, o.z);
                h1 = true;
            }
        }
        if (h0) {
            acc[0][0] += r0.x; acc[0][1] += r0.y; acc[0][2] += r0.z; cnt[0] += 1.0f;
        }
        if (h1) {
            acc[1][0] += r1.x; acc[1][1] += r1.y; acc[1][2] += r1.z; cnt[1] += 1.0f;
        }
        if (HITDIST) {
            const size_t rec = (size_t)p * a.rpp + k;
            const float l0 = __ldcs(a.ray_len + rec), l1 = __ldcs(a.ray_len + rec + 32);
            if (h0 && isfinite(l0) && l0 >= 0.0f) { hs[0] += l0; hn[0] += 1.0f; }
            if (h1 && isfinite(l1) && l1 >= 0.0f) { hs[1] += l1; hn[1] += 1.0f; }
        }
    }
    // cell means, then the radiance backup: cells without sample take the mean of populated cells
    float pop[4] = {0.f, 0.f, 0.f, 0.f};
    for (int h = 0; h < 2; ++h) {
        const float inv = cnt[h] > 0.f ? 1.0f / cnt[h] : 0.0f;
        for (int c = 0; c < 3; ++c) {
            L[h][c] = acc[h][c] * inv;
            pop[c] += L[h][c];
        }
        pop[3] += cnt[h] > 0.f ? 1.0f : 0.0f;
    }
    for (int o = 16; o; o >>= 1)
        for (int c = 0; c < 4; ++c) pop[c] += __shfl_xor_sync(kFullMask, pop[c], o);
    const float binv = pop[3] > 0.f ? 1.0f / pop[3] : 0.0f;
    for (int h = 0; h < 2; ++h)
        if (cnt[h] == 0.f)
            for (int c = 0; c < 3; ++c) L[h][c] = pop[c] * binv;
    for (int h = 0; h < 2; ++h) hd[h] = hn[h] > 0.f ? hs[h] / hn[h] : INFINITY;
}

// SH coefficients of channel h (coefficient k at out[3 k + h]) from the channel's ten direction
// moments Sc (local frame: solid angle, first moment xyz, second moment xx yy zz xy xz yz), rotated
// to world space by the probe frame of normal n4.
__device__ __forceinline__ void project_channel(const float4 n4, const float (&Sc)[10], int h, float *out) {
    // probe frame (Duff et al. 2017): columns t, b, n of R
    const float nx = n4.x, ny = n4.y, nz = n4.z;
    const float sgn = copysignf(1.0f, nz);
    const float ia = -1.0f / (sgn + nz);
    const float bb = nx * ny * ia;
    const float R[3][3] = {{1.0f + sgn * nx * nx * ia, bb, nx},
                           {sgn * bb, sgn + ny * ny * ia, ny},
                           {-sgn * nx, -ny, nz}};
    const float S0 = Sc[0];
    const float S1[3] = {Sc[1], Sc[2], Sc[3]};
    float S2[3][3];
    S2[0][0] = Sc[4]; S2[1][1] = Sc[5]; S2[2][2] = Sc[6];
    S2[0][1] = S2[1][0] = Sc[7];
    S2[0][2] = S2[2][0] = Sc[8];
    S2[1][2] = S2[2][1] = Sc[9];
    float W1[3], T[3][3], W2[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) W1[i] = R[i][0] * S1[0] + R[i][1] * S1[1] + R[i][2] * S1[2];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int q = 0; q < 3; ++q) T[i][q] = R[i][0] * S2[0][q] + R[i][1] * S2[1][q] + R[i][2] * S2[2][q];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) W2[i][j] = W2[j][i] = T[i][0] * R[j][0] + T[i][1] * R[j][1] + T[i][2] * R[j][2];
    // real SH basis, bands 0..2: c0; c1 y, c1 z, c1 x; c2 xy, c2 yz, c3 (3z^2 - 1), c2 xz, c4 (x^2 - y^2);
    // channel h, coefficient k at 3 k + h
    const float C0 = 0.28209479177387814f, C1 = 0.4886025119029199f, C2 = 1.0925484305920792f,
                C3 = 0.31539156525252005f, C4 = 0.5462742152960396f;
    out[0 * 3 + h] = C0 * S0;
    out[1 * 3 + h] = C1 * W1[1];
    out[2 * 3 + h] = C1 * W1[2];
    out[3 * 3 + h] = C1 * W1[0];
    out[4 * 3 + h] = C2 * W2[0][1];
    out[5 * 3 + h] = C2 * W2[1][2];
    out[6 * 3 + h] = C3 * (3.0f * W2[2][2] - S0);
    out[7 * 3 + h] = C2 * W2[0][2];
    out[8 * 3 + h] = C4 * (W2[0][0] - W2[1][1]);
}

// Probe irradiance (Sections 2.1.4, 2.4.2) with four threads per probe: thread h of a probe's quad
// takes the cells c = 16 h + i, i < 16, their slot ids in four 16-byte loads, and gathers their
// radiance kIntPass cells at a time; a cell's radiance is the mean of its rays that produced a sample, and the cell's exact
// direction moments (shared memory, 12 floats per cell: three 16-byte reads) are added in with
// multiply-adds.  Cells without sample take the mean of the populated cells (radiance backup)
// through the summed moments of the empty cells, the same sum by linearity.  Two xor-shuffle steps
// add the quad's partial moments; thread h < 3 then projects channel h.  (1080p: one warp per probe
// with a 31-shuffle reduce-scatter ran 31 us at ~600 instructions per probe; one thread per probe,
// 41 us: too few warps to hide the gathers.)  RPC1: one ray per cell.
constexpr int kIntThreads = 128;  // 32 probes per block
constexpr int kMomStride = 12;    // floats per cell in the shared moment table
constexpr int kIntPass = 8;       // cells per thread whose loads are in flight together

// Entry 4 i + h of the table holds cell 16 h + i, the i-th cell of thread h: the four threads of a
// quad read four entries 48 bytes apart (distinct banks).
__device__ __forceinline__ void load_moment_table(float *s_mom) {
    for (int k = threadIdx.x; k < 64 * kMomStride; k += blockDim.x) {
        const int e = k / kMomStride, m = k - e * kMomStride;
        const int c = 16 * (e & 3) + (e >> 2);
        s_mom[k] = m < 10 ? g_moments[m][c] : 0.0f;
    }
}

template <bool SURR, bool RPC1>
__device__ __forceinline__ void integrate_quad(const IntegrateArgs &a, uint32_t p, bool valid, const float *s_mom) {
    const int h = threadIdx.x & 3;
    float4 n4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) n4 = __ldg(a.nrm + p);
    const bool live = valid && n4.w != 0.0f;
    float S[10][3], U[10];
#pragma unroll
    for (int m = 0; m < 10; ++m) {
        S[m][0] = S[m][1] = S[m][2] = 0.0f;
        U[m] = 0.0f;
    }
    float pop0 = 0.f, pop1 = 0.f, pop2 = 0.f, npop = 0.f;
    if (live) {
        const uint32_t rpc = RPC1 ? 1u : (a.rpp >> 6);
        const size_t rec_base = (size_t)p * a.rpp;
        // thread h's 16 cells are consecutive: their slot ids come in four 16-byte loads
        const uint4 *ids = reinterpret_cast<const uint4 *>(a.slot_ids + rec_base + 16u * h);
        uint4 idq[4];
        if (RPC1) {
#pragma unroll
            for (int q = 0; q < 4; ++q) idq[q] = __ldcs(ids + q);
        }
#pragma unroll
        for (int i0 = 0; i0 < 16; i0 += kIntPass) {
            float acc[kIntPass][3], cnt[kIntPass];
#pragma unroll
            for (int i = 0; i < kIntPass; ++i) {
                acc[i][0] = acc[i][1] = acc[i][2] = 0.0f;
                cnt[i] = 0.0f;
            }
            for (uint32_t j = 0; j < rpc; ++j) {
                uint32_t sl[kIntPass];
                if (RPC1) {
#pragma unroll
                    for (int q = 0; q < kIntPass / 4; ++q) {
                        sl[4 * q + 0] = idq[i0 / 4 + q].x;
                        sl[4 * q + 1] = idq[i0 / 4 + q].y;
                        sl[4 * q + 2] = idq[i0 / 4 + q].z;
                        sl[4 * q + 3] = idq[i0 / 4 + q].w;
                    }
                } else {
                    const uint32_t *row = a.slot_ids + rec_base + j * 64u + 16u * h + i0;
#pragma unroll
                    for (int i = 0; i < kIntPass; ++i) sl[i] = __ldcs(row + i);
                }
                float3 r[kIntPass];
                bool hs[kIntPass];
#pragma unroll
                for (int i = 0; i < kIntPass; ++i) hs[i] = ray_sample(a, sl[i], r[i]);
                if (SURR) {
                    // records rec0 + i, rec0 = (p rpp + 64 j + 16 h + i0): bits 16 (h & 1) + i0 + i of
                    // the answer word of the 32 records starting at the probe's 64 j + 32 (h >> 1)
                    const size_t rec0 = rec_base + j * 64u + 16u * h + i0;
                    const uint32_t wbits = __ldg(a.ovr_bits + (rec0 >> 5)) >> ((rec0 & 31u));
#pragma unroll
                    for (int i = 0; i < kIntPass; ++i)
                        if ((wbits >> i) & 1u) {
                            const float4 o = __ldg(a.ovr + rec0 + i);
                            r[i] = make_float3(o.x, o.y, o.z);
                            hs[i] = true;
                        }
                }
#pragma unroll
                for (int i = 0; i < kIntPass; ++i)
                    if (hs[i]) {
                        acc[i][0] += r[i].x;
                        acc[i][1] += r[i].y;
                        acc[i][2] += r[i].z;
                        cnt[i] += 1.0f;
                    }
            }
#pragma unroll
            for (int i = 0; i < kIntPass; ++i) {
                const float4 *mc = reinterpret_cast<const float4 *>(s_mom + (4 * (i0 + i) + h) * kMomStride);
                const float4 w0 = mc[0], w1 = mc[1], w2 = mc[2];
                const float w[10] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w, w2.x, w2.y};
                if (cnt[i] > 0.0f) {
                    const float inv = RPC1 ? 1.0f : __frcp_rn(cnt[i]);
                    const float L0 = acc[i][0] * inv, L1 = acc[i][1] * inv, L2 = acc[i][2] * inv;
                    pop0 += L0;
                    pop1 += L1;
                    pop2 += L2;
                    npop += 1.0f;
#pragma unroll
                    for (int m = 0; m < 10; ++m) {
                        S[m][0] = fmaf(L0, w[m], S[m][0]);
                        S[m][1] = fmaf(L1, w[m], S[m][1]);
                        S[m][2] = fmaf(L2, w[m], S[m][2]);
                    }
                } else {
#pragma unroll
                    for (int m = 0; m < 10; ++m) U[m] += w[m];
                }
            }
        }
    }
    // the quad's partial sums (every lane takes part: the shuffles span the warp)
#pragma unroll
    for (int d = 1; d <= 2; d <<= 1) {
#pragma unroll
        for (int m = 0; m < 10; ++m) {
            S[m][0] += __shfl_xor_sync(kFullMask, S[m][0], d);
            S[m][1] += __shfl_xor_sync(kFullMask, S[m][1], d);
            S[m][2] += __shfl_xor_sync(kFullMask, S[m][2], d);
            U[m] += __shfl_xor_sync(kFullMask, U[m], d);
        }
        pop0 += __shfl_xor_sync(kFullMask, pop0, d);
        pop1 += __shfl_xor_sync(kFullMask, pop1, d);
        pop2 += __shfl_xor_sync(kFullMask, pop2, d);
        npop += __shfl_xor_sync(kFullMask, npop, d);
    }
    if (!valid) return;
    float *out = a.sh + (size_t)p * GI_SH_STRIDE;
    if (!live) {
        for (int k = h; k < GI_SH_STRIDE; k += 4) out[k] = 0.0f;
        return;
    }
    if (h == 3) {
        out[27] = 0.0f;
        return;
    }
    // radiance backup: every cell without sample holds the mean of the populated cells
    const float binv = npop > 0.0f ? 1.0f / npop : 0.0f;
    const float bk = (h == 0 ? pop0 : (h == 1 ? pop1 : pop2)) * binv;
    float Sc[10];
#pragma unroll
    for (int m = 0; m < 10; ++m) Sc[m] = fmaf(bk, U[m], h == 0 ? S[m][0] : (h == 1 ? S[m][1] : S[m][2]));
    project_channel(n4, Sc, h, out);
}

// blk: block of kIntThreads / 4 probes (the batched pass passes the view-local block).  RPC1: 64
// rays per probe (one per cell), a kernel of its own so that the general form's registers do not
// weigh on it.
template <bool SURR, bool RPC1>
__device__ __forceinline__ void integrate_body(const IntegrateArgs &a, uint32_t blk, const float *s_mom) {
    const uint32_t p = blk * (blockDim.x >> 2) + (threadIdx.x >> 2);
    integrate_quad<SURR, RPC1>(a, p, p < a.probes, s_mom);
}

template <bool RPC1>
__global__ void __launch_bounds__(kIntThreads, 4) k_integrate(IntegrateArgs a) {
    __shared__ __align__(16) float s_mom[64 * kMomStride];
    load_moment_table(s_mom);
    __syncthreads();
    integrate_body<false, RPC1>(a, blockIdx.x, s_mom);
}

// Probe atlas: float4 per (probe, cell) = (mean radiance rgb, mean hit distance); zeros for no probe.
__global__ void __launch_bounds__(256) k_gather(IntegrateArgs a, float4 *atlas) {
    const uint32_t p = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= a.probes) return;
    float4 *dst = atlas + (size_t)p * 64;
    if (__ldg(a.nrm + p).w == 0.0f) {
        dst[lane] = make_float4(0.f, 0.f, 0.f, 0.f);
        dst[lane + 32] = make_float4(0.f, 0.f, 0.f, 0.f);
        return;
    }
    float L[2][3], hd[2];
    gather_cells<false, true>(a, p, lane, L, hd);
    dst[lane] = make_float4(L[0][0], L[0][1], L[0][2], hd[0]);
    dst[lane + 32] = make_float4(L[1][0], L[1][1], L[1][2], hd[1]);
}

// SH coefficients of every probe from its atlas, four threads per probe as in the probe pass:
// thread h reads the consecutive cells 16 h + i (eight 16-byte loads in flight at a time) and adds
// each cell's radiance times its direction moments (shared table); two xor-shuffle steps add the
// quad's moments, then thread h < 3 projects channel h.  (1080p: one warp per probe with a
// 31-shuffle reduce-scatter took 19.5 us.)
constexpr int kProjThreads = 128;  // 32 probes per block
__global__ void __launch_bounds__(kProjThreads) k_project(const float4 *atlas, const float4 *nrm, float *sh,
                                                          uint32_t probes) {
    __shared__ __align__(16) float s_mom[64 * kMomStride];
    load_moment_table(s_mom);
    __syncthreads();
    const uint32_t p = blockIdx.x * (kProjThreads / 4) + (threadIdx.x >> 2);
    const int h = threadIdx.x & 3;
    const bool valid = p < probes;
    float4 n4 = make_float4(0.f, 0.f, 0.f, 0.f);
    if (valid) n4 = __ldg(nrm + p);
    const bool live = valid && n4.w != 0.0f;
    float S[10][3];
#pragma unroll
    for (int m = 0; m < 10; ++m) S[m][0] = S[m][1] = S[m][2] = 0.0f;
    if (live) {
        const float4 *src = atlas + (size_t)p * 64 + 16 * h;
#pragma unroll
        for (int i0 = 0; i0 < 16; i0 += 8) {
            float4 L[8];
#pragma unroll
            for (int i = 0; i < 8; ++i) L[i] = __ldg(src + i0 + i);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const float4 *mc = reinterpret_cast<const float4 *>(s_mom + (4 * (i0 + i) + h) * kMomStride);
                const float4 w0 = mc[0], w1 = mc[1], w2 = mc[2];
                const float w[10] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w, w2.x, w2.y};
#pragma unroll
                for (int m = 0; m < 10; ++m) {
                    S[m][0] = fmaf(L[i].x, w[m], S[m][0]);
                    S[m][1] = fmaf(L[i].y, w[m], S[m][1]);
                    S[m][2] = fmaf(L[i].z, w[m], S[m][2]);
                }
            }
        }
    }
    // the quad's partial sums (every lane takes part: the shuffles span the warp)
#pragma unroll
    for (int d = 1; d <= 2; d <<= 1)
#pragma unroll
        for (int m = 0; m < 10; ++m) {
            S[m][0] += __shfl_xor_sync(kFullMask, S[m][0], d);
            S[m][1] += __shfl_xor_sync(kFullMask, S[m][1], d);
            S[m][2] += __shfl_xor_sync(kFullMask, S[m][2], d);
        }
    if (!valid) return;
    float *out = sh + (size_t)p * GI_SH_STRIDE;
    if (!live) {
        for (int k = h; k < GI_SH_STRIDE; k += 4) out[k] = 0.0f;
        return;
    }
    if (h == 3) {
        out[27] = 0.0f;
        return;
    }
    float Sc[10];
#pragma unroll
    for (int m = 0; m < 10; ++m) Sc[m] = h == 0 ? S[m][0] : (h == 1 ? S[m][1] : S[m][2]);
    project_channel(n4, Sc, h, out);
}
template <bool RPC1>
__global__ void __launch_bounds__(kIntThreads, 4) k_integrate_surr(IntegrateArgs a) {
    __shared__ __align__(16) float s_mom[64 * kMomStride];
    load_moment_table(s_mom);
    __syncthreads();
    integrate_body<true, RPC1>(a, blockIdx.x, s_mom);
}

// ---------------------------------------------------------------- temporal path
constexpr uint32_t kScoreNone = (0x7BFFu << 16) | 0xFFFFu;  // half(65504) << 16 | 0xFFFF

__device__ __forceinline__ float dot3_rn(float ax, float ay, float az, float bx, float by, float bz) {
    return __fadd_rn(__fadd_rn(__fmul_rn(ax, bx), __fmul_rn(ay, by)), __fmul_rn(az, bz));
}

// Algorithm 1: four 8x8 tiles per block (one thread per pixel, lane = 8 ly + lx).  A pixel whose
// previous position q falls on a previous probe that lies within cell_size of the pixel's plane
// and faces within 0.95 of its normal bids (half(distance) << 16 | lane); the smallest bid places
// the tile's probe on its pixel, carrying that previous probe.
__global__ void __launch_bounds__(256) k_reproject(ReprojArgs a) {
    __shared__ uint32_t s_score[4];
    const uint32_t tl = threadIdx.x >> 6, lane = threadIdx.x & 63;
    const uint32_t t = blockIdx.x * 4u + tl;
    const uint32_t tx = t % a.tiles_x, ty = t / a.tiles_x;
    if (lane == 0) s_score[tl] = kScoreNone;
    __syncthreads();
    const uint32_t x = 8u * tx + (lane & 7u), y = 8u * ty + (lane >> 3);
    uint32_t my = kScoreNone, tq = 0;
    float3 w = make_float3(0.f, 0.f, 0.f);
    float4 nd = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ty < a.tiles_y && x < a.width && y < a.height) {
        nd = __ldg(a.gbuf + (size_t)y * a.width + x);
        if (isfinite(nd.w) && nd.w >= 0.0f) {
            const float2 mv = __ldg(a.motion + (size_t)y * a.width + x);
            const float fx = floorf(__fadd_rn(__fadd_rn((float)x, 0.5f), mv.x));
            const float fy = floorf(__fadd_rn(__fadd_rn((float)y, 0.5f), mv.y));
            if (fx >= 0.0f && fy >= 0.0f && fx < (float)a.width && fy < (float)a.height) {
                tq = ((uint32_t)fy >> 3) * a.tiles_x + ((uint32_t)fx >> 3);
                if (__ldg(a.prev_mask + tq) != GI_PROBE_NONE) {
                    w = pixel_world_exact(a.cam, x, y, nd.w);
                    const float4 pp = __ldg(a.prev_pos + tq), pn = __ldg(a.prev_nrm + tq);
                    const float vx = __fsub_rn(pp.x, w.x), vy = __fsub_rn(pp.y, w.y), vz = __fsub_rn(pp.z, w.z);
                    const float plane = fabsf(dot3_rn(vx, vy, vz, nd.x, nd.y, nd.z));
                    const float ncheck = dot3_rn(pn.x, pn.y, pn.z, nd.x, nd.y, nd.z);
                    if (plane < __fmul_rn(a.dscale, nd.w) && ncheck > 0.95f) {
                        const float dist = __fsqrt_rn(dot3_rn(vx, vy, vz, vx, vy, vz));
                        my = ((uint32_t)__half_as_ushort(__float2half_rn(dist)) << 16) | lane;
                        atomicMin(&s_score[tl], my);
                    }
                }
            }
        }
    }
    __syncthreads();
    if (ty >= a.tiles_y) return;
    const uint32_t best = s_score[tl];
    if (best == kScoreNone) {
        if (lane == 0) {
            a.mask[t] = GI_PROBE_NONE;
            a.pos[t] = make_float4(0.f, 0.f, 0.f, 0.f);
            a.nrm[t] = make_float4(0.f, 0.f, 0.f, 0.f);
            a.src[t] = GI_PROBE_NONE;
        }
    } else if (my == best) {
        a.mask[t] = (y << 16) | x;
        a.pos[t] = make_float4(w.x, w.y, w.z, nd.w);
        a.nrm[t] = make_float4(nd.x, nd.y, nd.z, 1.0f);
        a.src[t] = tq;
    }
}

// Algorithm 4 on one cell: alpha from the normalised luminance difference, squared after the clamp.
__device__ __forceinline__ float3 temporal_blend(float3 c, float3 p) {
    const float l1 = (c.x + c.y + c.z) * (1.0f / 3.0f);
    const float l2 = (p.x + p.y + p.z) * (1.0f / 3.0f);
    float al = fmaxf(l1 - l2 - fminf(l1, l2), 0.0f) / fmaxf(fmaxf(l1, l2), 1e-4f);
    al = fminf(fmaxf(al, 0.0f), 0.95f);
    al *= al;
    return make_float3(c.x + al * (p.x - c.x), c.y + al * (p.y - c.y), c.z + al * (p.z - c.z));
}

// One warp per 8x8 tile: a fresh probe gathers its spawn tile's rays (the cells' radiance and hit
// distance, as k_gather) and blends each cell with the same cell of the tile's reprojected probe;
// a reprojected-only probe copies its source's cells; a tile without probe gets zeros.
__global__ void __launch_bounds__(256) k_gather_temporal(TemporalArgs a) {
    const uint32_t t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= a.probes) return;
    const uint32_t tx = t % a.tiles_x, ty = t / a.tiles_x;
    const uint32_t st = 8u * a.upscale, sx = tx / a.upscale, sy = ty / a.upscale;
    const uint32_t px = min(st * sx + (uint32_t)a.jx, a.width - 1u);
    const uint32_t py = min(st * sy + (uint32_t)a.jy, a.height - 1u);
    bool fresh = false;
    if ((px >> 3) == tx && (py >> 3) == ty) {
        const float d = __ldg(&a.gbuf[(size_t)py * a.width + px].w);
        fresh = isfinite(d) && d >= 0.0f;
    }
    const uint32_t src = __ldg(a.src + t);
    float4 *dst = a.atlas + (size_t)t * 64;
    float4 o0 = make_float4(0.f, 0.f, 0.f, 0.f), o1 = o0;
    if (fresh) {
        float L[2][3], hd[2];
        gather_cells<false, true>(a.g, sy * a.spawn_x + sx, lane, L, hd);
        float3 c0 = make_float3(L[0][0], L[0][1], L[0][2]), c1 = make_float3(L[1][0], L[1][1], L[1][2]);
        if (src != GI_PROBE_NONE) {
            const float4 p0 = __ldg(a.prev_atlas + (size_t)src * 64 + lane);
            const float4 p1 = __ldg(a.prev_atlas + (size_t)src * 64 + lane + 32);
            c0 = temporal_blend(c0, make_float3(p0.x, p0.y, p0.z));
            c1 = temporal_blend(c1, make_float3(p1.x, p1.y, p1.z));
        }
        o0 = make_float4(c0.x, c0.y, c0.z, hd[0]);
        o1 = make_float4(c1.x, c1.y, c1.z, hd[1]);
    } else if (src != GI_PROBE_NONE) {
        o0 = __ldg(a.prev_atlas + (size_t)src * 64 + lane);
        o1 = __ldg(a.prev_atlas + (size_t)src * 64 + lane + 32);
    }
    dst[lane] = o0;
    dst[lane + 32] = o1;
}

// ---------------------------------------------------------------- interpolation

// Algorithm 3 from MIP level m0 on: probe-space position (tx, ty) at that level plus the
// offset; climb the chain (halving the position, floor) until a probe is found or the position
// leaves the level.
__device__ __forceinline__ uint32_t find_closest_probe(const uint32_t *mask, const MipInfo &mi, int tx, int ty, int ox,
                                                       int oy, int m0) {
#pragma unroll
    for (int m = 1; m < GI_MAX_MIPS; ++m) {
        if (m < m0) continue;
        if (m >= mi.count) break;
        const int x = tx + ox, y = ty + oy;
        if (x < 0 || y < 0 || x >= mi.w[m] || y >= mi.h[m]) break;
        const uint32_t p = __ldg(mask + mi.off[m] + y * mi.w[m] + x);
        if (p != GI_PROBE_NONE) return p;
        tx >>= 1;
        ty >>= 1;
    }
    return GI_PROBE_NONE;
}

__device__ __forceinline__ uint32_t pick_u4(const uint32_t (&v)[4], int i) {
    return i == 0 ? v[0] : (i == 1 ? v[1] : (i == 2 ? v[2] : v[3]));
}

// Per-warp copy of the four neighbours' data in shared memory: SH coefficients (27 + pad, seven
// float4), the position relative to the camera t_q d_q and the normal.
struct InterpNb {
    float4 c[4][7];
    float4 pos[4];
    float4 nrm[4];
    float4 eu[4];  // uniform warp: neighbour o's irradiance (xyz) and plane term (w)
    float4 n8;     // uniform warp: the four normal weights
};

// Terms of neighbour o for a pixel with normal n: its distance along n from the camera,
// (t_q d_q) . n, and the normal weight max(0, n . n_q)^8.
__device__ __forceinline__ void nb_terms(const InterpNb &s, int o, float nx, float ny, float nz, float &qn, float &n8) {
    const float4 P = s.pos[o], N = s.nrm[o];
    qn = P.x * nx + P.y * ny + P.z * nz;
    const float d = fmaxf(nx * N.x + ny * N.y + nz * N.z, 0.0f);
    const float d2 = d * d, d4 = d2 * d2;
    n8 = d4 * d4;
}

// E_q(n) of neighbour o: sum_k A_l Y_k(n) c_qk (coefficient 3 k + channel), read four at a time.
__device__ __forceinline__ void nb_irradiance(const InterpNb &s, int o, const float (&Yb)[9], float (&E)[3]) {
    E[0] = E[1] = E[2] = 0.f;
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        const float4 v = s.c[o][k];
        const float t[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (4 * k + j < 27) E[(4 * k + j) % 3] += Yb[(4 * k + j) / 3] * t[j];
    }
}

// A_l Y_lm(n) for the 9 coefficients of bands 0..2.
__device__ __forceinline__ void sh_lobe(float nx, float ny, float nz, float (&Yb)[9]) {
    const float PI = 3.14159265358979f;
    const float A0 = PI, A1 = 2.0f * PI / 3.0f, A2 = 0.25f * PI;
    Yb[0] = A0 * 0.28209479177387814f;
    Yb[1] = A1 * 0.4886025119029199f * ny;
    Yb[2] = A1 * 0.4886025119029199f * nz;
    Yb[3] = A1 * 0.4886025119029199f * nx;
    Yb[4] = A2 * 1.0925484305920792f * nx * ny;
    Yb[5] = A2 * 1.0925484305920792f * ny * nz;
    Yb[6] = A2 * 0.31539156525252005f * (3.0f * nz * nz - 1.0f);
    Yb[7] = A2 * 1.0925484305920792f * nx * nz;
    Yb[8] = A2 * 0.5462742152960396f * (nx * nx - ny * ny);
}

// One pixel of the interpolation: weights of the four neighbours (bilinear x normal x plane
// distance) and the weighted irradiance, or the relaxed / none / sky flags.  (fx, fy) is the
// pixel's bilinear position between the neighbours.  UNIFORM: the neighbours' irradiance and
// plane and normal terms were evaluated once for the warp (s.eu, s.n8); otherwise each is
// evaluated for this pixel's normal from the warp's shared copy.
template <bool UNIFORM>
__device__ __forceinline__ void interp_pixel(const InterpArgs &a, const InterpNb &s, int x, int y, float fx, float fy,
                                             const float4 nd, size_t pix, bool inb, bool act, const uint32_t (&q)[4]) {
    if (!inb) return;
    if (!act) {
        __stcs(a.out + pix, make_float4(0.f, 0.f, 0.f, (float)GI_INTERP_SKY));
        return;
    }
    const float nx = nd.x, ny = nd.y, nz = nd.z;
    // Plane distance of neighbour q from the pixel's plane, relative to the camera (the camera
    // origin cancels): (P_q - P_p) . n_p = (t_q d_q) . n_p - t_p (d_p . n_p).
    const float3 d = cam_ray_dir(a.cam, (float)x, (float)y);
    // (products rounded on their own: no contraction into the differences below, so that every
    // kernel instantiating this body rounds alike)
    const float pn = __fmul_rn(nd.w, d.x * nx + d.y * ny + d.z * nz);
    // the plane weight max(1 - |plane distance| / cs, 0) is taken times cs, which cancels in
    // es / wsum and keeps the sign of every weight
    const float cs = __fmul_rn(a.dscale, nd.w);
    float Yb[9];
    if (!UNIFORM) sh_lobe(nx, ny, nz, Yb);
    float wsum = 0.f, es[3] = {0.f, 0.f, 0.f};
    int nfound = 0;
#pragma unroll
    for (int o = 0; o < 4; ++o) {
        if (q[o] == GI_PROBE_NONE) continue;
        float qn, n8, E[3];
        if (UNIFORM) {
            const float4 u = s.eu[o];
            const float4 n8v = s.n8;
            qn = u.w;
            n8 = o == 0 ? n8v.x : (o == 1 ? n8v.y : (o == 2 ? n8v.z : n8v.w));
            E[0] = u.x;
            E[1] = u.y;
            E[2] = u.z;
        } else {
            nb_terms(s, o, nx, ny, nz, qn, n8);
            nb_irradiance(s, o, Yb, E);
        }
        const float bil = ((o & 1) ? fx : 1.0f - fx) * ((o >> 1) ? fy : 1.0f - fy);
        const float wd = fmaxf(cs - fabsf(qn - pn), 0.0f);
        const float w = bil * n8 * wd;
        wsum += w;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) es[ch] += w * E[ch];
        ++nfound;
    }
    float4 r;
    if (nfound == 0) {
        r = make_float4(0.f, 0.f, 0.f, (float)GI_INTERP_NONE);
    } else if (wsum > 0.0f) {
        const float inv = 1.0f / wsum;
        r = make_float4(es[0] * inv, es[1] * inv, es[2] * inv, (float)GI_INTERP_OK);
    } else {
        // relaxed: the plain mean of the neighbours found (rare: every weight vanished)
        float er[3] = {0.f, 0.f, 0.f};
#pragma unroll
        for (int o = 0; o < 4; ++o) {
            if (q[o] == GI_PROBE_NONE) continue;
            float E[3];
            if (UNIFORM) {
                const float4 u = s.eu[o];
                E[0] = u.x;
                E[1] = u.y;
                E[2] = u.z;
            } else {
                nb_irradiance(s, o, Yb, E);
            }
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) er[ch] += E[ch];
        }
        const float inv = 1.0f / (float)nfound;
        r = make_float4(er[0] * inv, er[1] * inv, er[2] * inv, (float)GI_INTERP_RELAXED);
    }
    __stcs(a.out + pix, r);
}

constexpr int kInterpWarps = 8;  // 32 x 16 pixels per 256-thread block

// Block = 32x16 pixels starting at (32 bx - 4, 16 by - 4); warp = the 8x8 pixels that share one
// base tile floor((p - 4) / 8): lane l holds column l & 7 of rows l >> 3 and 4 + (l >> 3).  The
// four neighbour probes are therefore the same for the whole warp: lanes 0..3 run Algorithm 3
// for one neighbour each, and the warp copies the neighbours' data to shared memory once (28 lanes
// one SH float4 each, 4 lanes a position and normal).  A warp whose active pixels share one normal
// evaluates the neighbours' irradiance and plane terms once for its 64 pixels.
__device__ __forceinline__ void interpolate_body(const InterpArgs &a, uint32_t bx, uint32_t by) {
    __shared__ InterpNb s_nb[kInterpWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    InterpNb &s = s_nb[warp];
    const int x = (int)bx * 32 - 4 + 8 * (warp & 3) + (lane & 7);
    const int y0 = (int)by * 16 - 4 + 8 * (warp >> 2) + (lane >> 3);
    const int tx = (x - 4) >> 3, ty = (y0 - 4) >> 3;  // the same for y0 and y0 + 4
    // the G-buffer of the lane's two pixels (independent of the probes)
    bool inb[2], act[2];
    float4 nd[2];
    size_t pix[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int y = y0 + 4 * h;
        inb[h] = x >= 0 && y >= 0 && x < (int)a.width && y < (int)a.height;
        pix[h] = inb[h] ? (size_t)y * a.width + x : 0;
        nd[h] = inb[h] ? __ldcs(a.gbuf + pix[h]) : make_float4(0.f, 0.f, 0.f, -1.0f);
    }
    // neighbour `lane` (lanes 0..3): Algorithm 3 from the tile (tx + (lane & 1), ty + (lane >> 1)),
    // continued above level 0 only where level 0 holds no probe
    uint32_t qo = GI_PROBE_NONE;
    if (lane < 4) {
        const int qx = tx + (lane & 1), qy = ty + (lane >> 1);
        if (qx >= 0 && qy >= 0 && qx < a.mi.w[0] && qy < a.mi.h[0]) {
            qo = __ldg(a.mask + qy * a.mi.w[0] + qx);
            if (qo == GI_PROBE_NONE) qo = find_closest_probe(a.mask, a.mi, tx >> 1, ty >> 1, lane & 1, lane >> 1, 1);
        }
    }
    uint32_t q[4];
#pragma unroll
    for (int o = 0; o < 4; ++o) q[o] = __shfl_sync(kFullMask, qo, o);
#pragma unroll
    for (int h = 0; h < 2; ++h) act[h] = inb[h] && isfinite(nd[h].w) && nd[h].w >= 0.0f;
    const unsigned am0 = __ballot_sync(kFullMask, act[0]), am1 = __ballot_sync(kFullMask, act[1]);
    if ((am0 | am1) == 0u) {  // the whole warp is sky or outside the image
#pragma unroll
        for (int h = 0; h < 2; ++h)
            if (inb[h]) __stcs(a.out + pix[h], make_float4(0.f, 0.f, 0.f, (float)GI_INTERP_SKY));
        return;
    }
    // the neighbours' data into the warp's shared copy
    {
        const int o = lane < 28 ? lane / 7 : lane - 28;
        const uint32_t qq = pick_u4(q, o);
        if (qq != GI_PROBE_NONE) {
            const uint32_t pidx = (qq >> 19) * a.tiles_x + ((qq & 0xFFFFu) >> 3);
            if (lane < 28) {
                const int k = lane - 7 * o;
                s.c[o][k] = __ldg(reinterpret_cast<const float4 *>(a.sh + (size_t)pidx * GI_SH_STRIDE) + k);
            } else {
                const float tq = __ldg(a.ppos + pidx).w;
                const float qpx = (float)(qq & 0xFFFFu), qpy = (float)(qq >> 16);
                const float sxq = (2.0f * (qpx + 0.5f) * a.cam.inv_w - 1.0f) * a.cam.sx_scale;
                const float syq = (1.0f - 2.0f * (qpy + 0.5f) * a.cam.inv_h) * a.cam.sy_scale;
                const float vx = a.cam.fwd[0] + sxq * a.cam.right[0] + syq * a.cam.up[0];
                const float vy = a.cam.fwd[1] + sxq * a.cam.right[1] + syq * a.cam.up[1];
                const float vz = a.cam.fwd[2] + sxq * a.cam.right[2] + syq * a.cam.up[2];
                const float t = tq * rsqrtf(vx * vx + vy * vy + vz * vz);
                s.pos[o] = make_float4(t * vx, t * vy, t * vz, 0.f);
                s.nrm[o] = __ldg(a.pnrm + pidx);
            }
        }
    }
    __syncwarp();
    // the first active pixel's normal stands in for inactive pixels (they only help the warp)
    const int src = __ffs(am0 ? am0 : am1) - 1;
    const float4 ns = am0 ? nd[0] : nd[1];
    const float sx_ = __shfl_sync(kFullMask, ns.x, src), sy_ = __shfl_sync(kFullMask, ns.y, src),
                sz_ = __shfl_sync(kFullMask, ns.z, src);
    bool same = true;
#pragma unroll
    for (int h = 0; h < 2; ++h)
        same = same && (!act[h] || (__float_as_uint(nd[h].x) == __float_as_uint(sx_) &&
                                    __float_as_uint(nd[h].y) == __float_as_uint(sy_) &&
                                    __float_as_uint(nd[h].z) == __float_as_uint(sz_)));
    const bool uniform = __all_sync(kFullMask, same);
    const float fx = ((float)(lane & 7) + 0.5f) * 0.125f;
    // uniform warp: lane 3 o + ch evaluates neighbour o, channel ch; lanes 12..15 the plane and
    // normal terms of neighbour lane - 12; the results go to the warp's shared copy
    if (uniform) {
        if (lane < 12) {
            const int o = lane / 3, ch = lane - 3 * (lane / 3);
            float e = 0.f;
            if (pick_u4(q, o) != GI_PROBE_NONE) {
                float Yb[9];
                sh_lobe(sx_, sy_, sz_, Yb);
                const float *c = reinterpret_cast<const float *>(s.c[o]) + ch;
#pragma unroll
                for (int k = 0; k < 9; ++k) e += Yb[k] * c[3 * k];
            }
            reinterpret_cast<float *>(s.eu)[4 * o + ch] = e;
        } else if (lane < 16) {
            const int o = lane - 12;
            float qn_u = 0.f, n8_u = 0.f;
            if (pick_u4(q, o) != GI_PROBE_NONE) nb_terms(s, o, sx_, sy_, sz_, qn_u, n8_u);
            reinterpret_cast<float *>(s.eu)[4 * o + 3] = qn_u;
            reinterpret_cast<float *>(&s.n8)[o] = n8_u;
        }
        __syncwarp();
#pragma unroll
        for (int h = 0; h < 2; ++h)
            interp_pixel<true>(a, s, x, y0 + 4 * h, fx, ((float)((lane >> 3) + 4 * h) + 0.5f) * 0.125f,
                               h ? nd[1] : nd[0], h ? pix[1] : pix[0], h ? inb[1] : inb[0], h ? act[1] : act[0], q);
    } else {
#pragma unroll 1
        for (int h = 0; h < 2; ++h)
            interp_pixel<false>(a, s, x, y0 + 4 * h, fx, ((float)((lane >> 3) + 4 * h) + 0.5f) * 0.125f,
                                h ? nd[1] : nd[0], h ? pix[1] : pix[0], h ? inb[1] : inb[0], h ? act[1] : act[0], q);
    }
}

__global__ void __launch_bounds__(256, 4) k_interpolate(InterpArgs a) { interpolate_body(a, blockIdx.x, blockIdx.y); }

static bool layout_matches(const gi_probe_layout &l, uint32_t w, uint32_t h) {
    return l.tiles_x == (w + 7) / 8 && l.tiles_y == (h + 7) / 8 && l.num_probes == l.tiles_x * l.tiles_y &&
           l.mip_count >= 1 && l.mip_count <= GI_MAX_MIPS;
}

static int halton_scaled(uint32_t i, uint32_t base, uint32_t scale) {
    // floor(scale * radical_inverse_base(i)) with exact integer arithmetic
    uint64_t num = 0, den = 1;
    while (i) {
        num = num * base + i % base;
        den *= base;
        i /= base;
    }
    return (int)((scale * num) / den);
}


gi_status spawn_check(const gi_gbuffer *gbuf, const gi_view *view, const gi_probes *pr) {
    if (!gbuf || !pr || !view_ok(view) || !gbuf->nd || !pr->mask || !pr->pos || !pr->nrm) {
        set_error("gi_probes_spawn: NULL argument or bad view");
        return GI_ERR_INVALID_ARG;
    }
    if (gbuf->width != view->width || gbuf->height != view->height ||
        !layout_matches(pr->layout, view->width, view->height) || ((uintptr_t)gbuf->nd & 15) ||
        ((uintptr_t)pr->pos & 15) || ((uintptr_t)pr->nrm & 15)) {
        set_error("gi_probes_spawn: G-buffer/probe layout does not match the view, or misaligned buffers");
        return GI_ERR_INVALID_ARG;
    }
    return GI_OK;
}

SpawnArgs spawn_args(const gi_gbuffer *gbuf, const gi_view *view, const gi_probes *pr) {
    SpawnArgs a;
    a.gbuf = reinterpret_cast<const float4 *>(gbuf->nd);
    a.width = view->width;
    a.height = view->height;
    a.cam = cam_params(view);
    a.jx = halton_scaled(view->frame + 1u, 2, 8u);
    a.jy = halton_scaled(view->frame + 1u, 3, 8u);
    a.upscale = 1u;
    a.keep = 0u;
    a.mask = pr->mask;
    a.pos = reinterpret_cast<float4 *>(pr->pos);
    a.nrm = reinterpret_cast<float4 *>(pr->nrm);
    a.tiles_x = pr->layout.tiles_x;
    a.tiles_y = pr->layout.tiles_y;
    a.mi = mip_info(pr->layout);
    return a;
}

gi_status integrate_check(gi_cache_t cache, const gi_probes *pr, const uint32_t *slot_ids, uint32_t rays_per_probe) {
    if (!cache || !pr || !pr->nrm || !pr->sh || (!slot_ids && pr->layout.num_probes > 0)) {
        set_error("gi_probes_integrate: NULL argument");
        return GI_ERR_INVALID_ARG;
    }
    if (rays_per_probe == 0 || rays_per_probe % 64 != 0 || ((uintptr_t)pr->nrm & 15) || ((uintptr_t)slot_ids & 15)) {
        set_error("gi_probes_integrate: rays_per_probe must be a positive multiple of 64; nrm and slot_ids 16-byte "
                  "aligned");
        return GI_ERR_INVALID_ARG;
    }
    return GI_OK;
}

IntegrateArgs integrate_args(gi_cache_t cache, const gi_probes *pr, const uint32_t *slot_ids, uint32_t rpp,
                             const float env[3]) {
    const CacheView cv = cache_view(cache);
    IntegrateArgs a;
    a.slot_ids = slot_ids;
    a.resolved = cv.resolved;
    a.res_stride = cv.resolved_stride;
    a.f16 = cv.resolved_f16;
    a.slots = cv.slots;
    a.nrm = reinterpret_cast<const float4 *>(pr->nrm);
    a.sh = pr->sh;
    a.probes = pr->layout.num_probes;
    a.rpp = rpp;
    for (int c = 0; c < 3; ++c) a.env[c] = env ? env[c] : 0.0f;
    a.ovr_bits = nullptr;
    a.ovr = nullptr;
    a.ray_len = nullptr;
    return a;
}

gi_status interp_check(const gi_gbuffer *gbuf, const gi_view *view, const gi_probes *pr, const float *out) {
    if (!gbuf || !pr || !out || !view_ok(view) || !gbuf->nd || !pr->mask || !pr->pos || !pr->nrm || !pr->sh) {
        set_error("gi_probes_interpolate: NULL argument or bad view");
        return GI_ERR_INVALID_ARG;
    }
    if (gbuf->width != view->width || gbuf->height != view->height ||
        !layout_matches(pr->layout, view->width, view->height) || ((uintptr_t)gbuf->nd & 15) ||
        ((uintptr_t)out & 15) || ((uintptr_t)pr->sh & 15)) {
        set_error("gi_probes_interpolate: layout does not match the view, or misaligned buffers");
        return GI_ERR_INVALID_ARG;
    }
    return GI_OK;
}

InterpArgs interp_args(const gi_gbuffer *gbuf, const gi_view *view, const gi_probes *pr, float *out) {
    InterpArgs a;
    a.gbuf = reinterpret_cast<const float4 *>(gbuf->nd);
    a.width = view->width;
    a.height = view->height;
    a.cam = cam_params(view);
    a.dscale = (float)distance_scale(view->fov_y, view->width, view->height);
    a.mask = pr->mask;
    a.mi = mip_info(pr->layout);
    a.ppos = reinterpret_cast<const float4 *>(pr->pos);
    a.pnrm = reinterpret_cast<const float4 *>(pr->nrm);
    a.sh = pr->sh;
    a.tiles_x = pr->layout.tiles_x;
    a.out = reinterpret_cast<float4 *>(out);
    return a;
}


// ---------------------------------------------------------------- probe filtering (Algorithm 5)

struct FilterArgs {
    const float4 *in;
    float4 *out;
    const uint32_t *mask;
    MipInfo mi;
    const float4 *ppos;  // xyz, distance along the pixel ray
    const float4 *pnrm;  // xyz, 1 = probe / 0 = none
    uint32_t probes, tiles_x;
    float dscale;        // Algorithm 6: cell_size(d) = dscale * d
    int axis;            // 0: steps along x, 1: along y
};

// Algorithm 3 from level 0: the probe at (tx + ox, ty + oy), else up the MIP chain.
__device__ __forceinline__ uint32_t find_probe_from_level0(const uint32_t *mask, const MipInfo &mi, int tx, int ty,
                                                            int ox, int oy) {
    const int x = tx + ox, y = ty + oy;
    if (x < 0 || y < 0 || x >= mi.w[0] || y >= mi.h[0]) return GI_PROBE_NONE;
    const uint32_t q = __ldg(mask + y * mi.w[0] + x);
    if (q != GI_PROBE_NONE) return q;
    return find_closest_probe(mask, mi, tx >> 1, ty >> 1, ox, oy, 1);
}

// One thread per (probe, cell), 4 probes per block (2 warps per probe): the cell's radiance and hit
// distance blurred with the same cell of the probes found at steps -1, +1, -2, +2, -3, +3 along the
// axis, each accepted when it lies within cell_size of the probe's plane, the cell direction is not
// behind its normal, and the hit point seen from it (at the smaller hit distance) is within pi/50 of
// the cell direction seen from the probe; depth weight 1 / (1 + |d_p - d_q| / cell_size(d_p)).
// What is the same for all 64 cells of a probe -- the neighbour search, its offset from the probe,
// the plane test and the depth weight -- lanes 0..5 of each warp compute once into shared memory;
// every thread then issues its six neighbour loads together and takes the per-cell decisions in
// step order (the running hit distance of one step enters the next).  The angle test avoids the
// square root: cos(angle) >= c  <=>  d.h > 0 and (d.h)^2 >= c^2 |h|^2.
constexpr int kFiltProbes = 4;
__global__ void __launch_bounds__(64 * kFiltProbes) k_filter(FilterArgs a) {
    __shared__ uint32_t s_qi[2 * kFiltProbes][6];
    __shared__ float4 s_rel[2 * kFiltProbes][6];  // q - p (xyz), depth weight
    __shared__ float4 s_nq[2 * kFiltProbes][6];
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const uint32_t p = blockIdx.x * kFiltProbes + (t >> 6);
    const uint32_t c = t & 63;
    if (p >= a.probes) return;  // both warps of a probe leave together
    const size_t self = (size_t)p * 64 + c;
    const float4 v = __ldg(a.in + self);
    const float4 n4 = __ldg(a.pnrm + p);
    if (n4.w == 0.0f) {
        a.out[self] = v;
        return;
    }
    const float4 pp = __ldg(a.ppos + p);
    const float cs = a.dscale * pp.w;
    const float nx = n4.x, ny = n4.y, nz = n4.z;
    if (lane < 6) {
        const int step = (((lane & 1) << 1) - 1) * ((lane >> 1) + 1);
        const int tx = (int)(p % a.tiles_x), ty = (int)(p / a.tiles_x);
        const uint32_t q = find_probe_from_level0(a.mask, a.mi, tx, ty, a.axis == 0 ? step : 0, a.axis == 0 ? 0 : step);
        uint32_t qi = GI_PROBE_NONE;
        if (q != GI_PROBE_NONE) {
            const uint32_t k = ((q >> 16) >> 3) * a.tiles_x + ((q & 0xFFFFu) >> 3);
            const float4 pq = __ldg(a.ppos + k);
            const float rx = pq.x - pp.x, ry = pq.y - pp.y, rz = pq.z - pp.z;
            if (fabsf(rx * nx + ry * ny + rz * nz) <= cs) {  // the plane test
                qi = k;
                s_rel[warp][lane] = make_float4(rx, ry, rz, __fdividef(cs, cs + fabsf(pp.w - pq.w)));
                s_nq[warp][lane] = __ldg(a.pnrm + k);
            }
        }
        s_qi[warp][lane] = qi;
    }
    __syncwarp();
    float4 vq[6];
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const uint32_t qi = s_qi[warp][i];
        vq[i] = qi != GI_PROBE_NONE ? __ldg(a.in + (size_t)qi * 64 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    // world direction of the cell centre in the probe frame (Duff et al. 2017)
    const float sgn = copysignf(1.0f, nz);
    const float ia = -1.0f / (sgn + nz);
    const float bb = nx * ny * ia;
    const float t0 = 1.0f + sgn * nx * nx * ia, t1 = sgn * bb, t2 = -sgn * nx;
    const float b0 = bb, b1 = sgn + ny * ny * ia, b2 = -ny;
    const float lx = __ldg(&g_cell_dir[c][0]), ly = __ldg(&g_cell_dir[c][1]), lz = __ldg(&g_cell_dir[c][2]);
    const float dx = lx * t0 + ly * b0 + lz * nx, dy = lx * t1 + ly * b1 + lz * ny, dz = lx * t2 + ly * b2 + lz * nz;
    const float cos2 = c_filter_cos * c_filter_cos;
    float r = v.x, gch = v.y, bch = v.z, acc_a = v.w, weight = 1.0f, hd = v.w;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        if (s_qi[warp][i] == GI_PROBE_NONE) continue;
        const float4 nq = s_nq[warp][i];
        if (dx * nq.x + dy * nq.y + dz * nq.z < 0.0f) continue;  // the cell points behind q
        const float4 rel = s_rel[warp][i];
        const float hdc = fminf(vq[i].w, hd);
        if (isfinite(hdc)) {
            const float hx = rel.x + dx * hdc, hy = rel.y + dy * hdc, hz = rel.z + dz * hdc;
            const float hh = hx * hx + hy * hy + hz * hz;
            const float dh = dx * hx + dy * hy + dz * hz;
            // a zero vector counts as on the cell direction
            if (hh > 0.0f && (dh <= 0.0f || dh * dh < cos2 * hh)) continue;
        }
        const float w = rel.w;
        r += w * vq[i].x;
        gch += w * vq[i].y;
        bch += w * vq[i].z;
        acc_a += w * hdc;
        weight += w;
        hd = __fdividef(acc_a, weight);
    }
    const float inv = __fdividef(1.0f, weight);
    a.out[self] = make_float4(r * inv, gch * inv, bch * inv, acc_a * inv);
}

// ---------------------------------------------------------------- batched passes (many views)
__global__ void __launch_bounds__(256) k_spawn_batched(const SpawnArgs *args, const uint32_t *prefix, uint32_t nviews) {
    __shared__ SpawnArgs sa;
    GI_BATCHED_ITEMS(prefix, nviews, sa, args, {
        const uint32_t gx = (sa.tiles_x + 15) / 16;
        spawn_body(sa, item % gx, item / gx);
    });
}

// MIP levels 5 and up of every view: one block per view.
__global__ void __launch_bounds__(1024) k_mip_tail_batched(const SpawnArgs *args) {
    __shared__ SpawnArgs sa;
    load_view_args(sa, args + blockIdx.x);
    __syncthreads();
    if (sa.mi.count > 5) mip_tail_body(sa.mask, sa.mi);
}

template <bool RPC1>
__global__ void __launch_bounds__(128, 4) k_integrate_batched(const IntegrateArgs *args, const uint32_t *prefix,
                                                           uint32_t nviews) {
    __shared__ IntegrateArgs sa;
    __shared__ __align__(16) float s_mom[64 * kMomStride];
    load_moment_table(s_mom);
    GI_BATCHED_ITEMS(prefix, nviews, sa, args, (integrate_body<false, RPC1>(sa, item, s_mom)));
}

__global__ void __launch_bounds__(256, 4) k_interpolate_batched(const InterpArgs *args, const uint32_t *prefix,
                                                                uint32_t nviews) {
    __shared__ InterpArgs sa;
    GI_BATCHED_ITEMS(prefix, nviews, sa, args, {
        const uint32_t gx = interp_grid_x(sa.width);
        interpolate_body(sa, item % gx, item / gx);
    });
}

gi_status launch_spawn_batched(const SpawnArgs *args, const uint32_t *prefix, uint32_t nviews, uint32_t blocks,
                               cudaStream_t st) {
    if (blocks == 0) return GI_OK;
    k_spawn_batched<<<resident_grid(k_spawn_batched, 256, blocks), 256, 0, st>>>(args, prefix, nviews);
    gi_status s = cuda_status(cudaGetLastError(), "k_spawn_batched launch");
    if (s != GI_OK) return s;
    k_mip_tail_batched<<<nviews, 1024, 0, st>>>(args);
    return cuda_status(cudaGetLastError(), "k_mip_tail_batched launch");
}

gi_status launch_integrate_batched(const IntegrateArgs *args, const uint32_t *prefix, uint32_t nviews,
                                   uint32_t blocks, uint32_t threads, uint32_t rays_per_probe, cudaStream_t st) {
    if (blocks == 0) return GI_OK;
    if (rays_per_probe == 64)
        k_integrate_batched<true><<<resident_grid(k_integrate_batched<true>, (int)threads, blocks), threads, 0, st>>>(
            args, prefix, nviews);
    else
        k_integrate_batched<false><<<resident_grid(k_integrate_batched<false>, (int)threads, blocks), threads, 0, st>>>(
            args, prefix, nviews);
    return cuda_status(cudaGetLastError(), "k_integrate_batched launch");
}

gi_status launch_interpolate_batched(const InterpArgs *args, const uint32_t *prefix, uint32_t nviews,
                                     uint32_t blocks, cudaStream_t st) {
    if (blocks == 0) return GI_OK;
    k_interpolate_batched<<<resident_grid(k_interpolate_batched, 256, blocks), 256, 0, st>>>(args, prefix, nviews);
    return cuda_status(cudaGetLastError(), "k_interpolate_batched launch");
}

} // namespace gi

using namespace gi;

extern "C" {

gi_status gi_cell_moments(double *out640) {
    if (!out640) {
        set_error("gi_cell_moments: out is NULL");
        return GI_ERR_INVALID_ARG;
    }
    for (int c = 0; c < 64; ++c) cell_moments_closed_form(c, out640 + 10 * c);
    return GI_OK;
}

gi_status gi_probes_layout(uint32_t width, uint32_t height, gi_probe_layout *out) {
    if (!out || width == 0 || height == 0 || width > 65535 || height > 65535) {
        set_error("gi_probes_layout: bad size or NULL output");
        return GI_ERR_INVALID_ARG;
    }
    memset(out, 0, sizeof *out);
    out->tiles_x = (width + 7) / 8;
    out->tiles_y = (height + 7) / 8;
    out->num_probes = out->tiles_x * out->tiles_y;
    uint32_t w = out->tiles_x, h = out->tiles_y, off = 0, k = 0;
    for (;;) {
        out->mip_w[k] = w;
        out->mip_h[k] = h;
        out->mip_offset[k] = off;
        off += w * h;
        ++k;
        if (w == 1 && h == 1) break;
        w = (w + 1) / 2;
        h = (h + 1) / 2;
    }
    out->mip_count = k;
    out->mask_words = off;
    return GI_OK;
}

gi_status gi_probes_spawn(const gi_gbuffer *gbuf, const gi_view *view, const gi_probes *pr, gi_stream_t stream) {
    gi_status s = spawn_check(gbuf, view, pr);
    if (s != GI_OK) return s;
    cudaStream_t st = (cudaStream_t)stream;
    const SpawnArgs a = spawn_args(gbuf, view, pr);
    dim3 grid((a.tiles_x + 15) / 16, (a.tiles_y + 15) / 16);
    k_spawn<<<grid, 256, 0, st>>>(a);
    s = cuda_status(cudaGetLastError(), "k_spawn launch");
    if (s == GI_OK && a.mi.count > 5) {
        k_mip_tail<<<1, 1024, 0, st>>>(pr->mask, a.mi);
        s = cuda_status(cudaGetLastError(), "k_mip_tail launch");
    }
    return s;
}

gi_status gi_probes_spawn_upscaled(const gi_gbuffer *gbuf, const gi_view *view, uint32_t upscale, uint32_t keep,
                                   const gi_probes *pr, gi_stream_t stream) {
    gi_status s = spawn_check(gbuf, view, pr);
    if (s != GI_OK) return s;
    if (upscale < 1 || upscale > GI_MAX_UPSCALE) {
        set_error("gi_probes_spawn_upscaled: upscale must be in 1..%d", GI_MAX_UPSCALE);
        return GI_ERR_INVALID_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    SpawnArgs a = spawn_args(gbuf, view, pr);
    a.upscale = upscale;
    a.keep = keep ? 1u : 0u;
    a.jx = halton_scaled(view->frame + 1u, 2, 8u * upscale);
    a.jy = halton_scaled(view->frame + 1u, 3, 8u * upscale);
    dim3 grid((a.tiles_x + 15) / 16, (a.tiles_y + 15) / 16);
    k_spawn<<<grid, 256, 0, st>>>(a);
    s = cuda_status(cudaGetLastError(), "k_spawn launch");
    if (s == GI_OK && a.mi.count > 5) {
        k_mip_tail<<<1, 1024, 0, st>>>(pr->mask, a.mi);
        s = cuda_status(cudaGetLastError(), "k_mip_tail launch");
    }
    return s;
}

gi_status gi_probes_reproject(const gi_gbuffer *gbuf, const gi_view *view, const float *motion,
                              const gi_probes *prev, const gi_probes *cur, uint32_t *src, gi_stream_t stream) {
    gi_status s = spawn_check(gbuf, view, cur);
    if (s != GI_OK) return s;
    if (!motion || !src || !prev || !prev->mask || !prev->pos || !prev->nrm || ((uintptr_t)motion & 7) ||
        ((uintptr_t)prev->pos & 15) || ((uintptr_t)prev->nrm & 15) ||
        prev->layout.num_probes != cur->layout.num_probes || prev->layout.tiles_x != cur->layout.tiles_x ||
        prev->mask == cur->mask || prev->pos == cur->pos || prev->nrm == cur->nrm) {
        set_error("gi_probes_reproject: NULL or misaligned argument, or prev and cur not two distinct probe "
                  "buffers of the same layout");
        return GI_ERR_INVALID_ARG;
    }
    ReprojArgs a;
    a.gbuf = reinterpret_cast<const float4 *>(gbuf->nd);
    a.motion = reinterpret_cast<const float2 *>(motion);
    a.width = view->width;
    a.height = view->height;
    a.tiles_x = cur->layout.tiles_x;
    a.tiles_y = cur->layout.tiles_y;
    a.cam = cam_params(view);
    a.dscale = (float)distance_scale(view->fov_y, view->width, view->height);
    a.prev_mask = prev->mask;
    a.prev_pos = reinterpret_cast<const float4 *>(prev->pos);
    a.prev_nrm = reinterpret_cast<const float4 *>(prev->nrm);
    a.mask = cur->mask;
    a.pos = reinterpret_cast<float4 *>(cur->pos);
    a.nrm = reinterpret_cast<float4 *>(cur->nrm);
    a.src = src;
    const uint32_t P = cur->layout.num_probes;
    k_reproject<<<(P + 3) / 4, 256, 0, (cudaStream_t)stream>>>(a);
    return cuda_status(cudaGetLastError(), "k_reproject launch");
}

gi_status gi_probes_gather_temporal(gi_cache_t cache, const gi_gbuffer *gbuf, const gi_view *view, uint32_t upscale,
                                    const gi_probes *pr, const uint32_t *slot_ids, const float *ray_len,
                                    uint32_t rays_per_probe, const uint32_t *src, const float *prev_atlas,
                                    float *atlas, const float env[3], gi_stream_t stream) {
    gi_status s = integrate_check(cache, pr, slot_ids, rays_per_probe);
    if (s != GI_OK) return s;
    if (!gbuf || !gbuf->nd || !view_ok(view) || gbuf->width != view->width || gbuf->height != view->height ||
        !layout_matches(pr->layout, view->width, view->height) || !ray_len || !src || !prev_atlas || !atlas ||
        prev_atlas == atlas || ((uintptr_t)prev_atlas & 15) || ((uintptr_t)atlas & 15) ||
        ((uintptr_t)gbuf->nd & 15) || upscale < 1 || upscale > GI_MAX_UPSCALE) {
        set_error("gi_probes_gather_temporal: NULL, aliased or misaligned buffer, size mismatch or bad upscale");
        return GI_ERR_INVALID_ARG;
    }
    TemporalArgs a;
    a.g = integrate_args(cache, pr, slot_ids, rays_per_probe, env);
    a.g.ray_len = ray_len;
    const uint32_t su = 8u * upscale;
    a.spawn_x = (view->width + su - 1) / su;
    a.g.probes = a.spawn_x * ((view->height + su - 1) / su);
    a.gbuf = reinterpret_cast<const float4 *>(gbuf->nd);
    a.width = view->width;
    a.height = view->height;
    a.tiles_x = pr->layout.tiles_x;
    a.probes = pr->layout.num_probes;
    a.upscale = upscale;
    a.jx = halton_scaled(view->frame + 1u, 2, su);
    a.jy = halton_scaled(view->frame + 1u, 3, su);
    a.src = src;
    a.prev_atlas = reinterpret_cast<const float4 *>(prev_atlas);
    a.atlas = reinterpret_cast<float4 *>(atlas);
    const uint32_t blocks = (a.probes + 7) / 8;
    if (blocks == 0) return GI_OK;
    k_gather_temporal<<<blocks, 256, 0, (cudaStream_t)stream>>>(a);
    return cuda_status(cudaGetLastError(), "k_gather_temporal launch");
}

gi_status gi_probes_integrate(gi_cache_t cache, const gi_probes *pr, const uint32_t *slot_ids,
                              uint32_t rays_per_probe, const float env[3], gi_stream_t stream) {
    gi_status s = integrate_check(cache, pr, slot_ids, rays_per_probe);
    if (s != GI_OK) return s;
    s = ensure_moments();
    if (s != GI_OK) return s;
    const IntegrateArgs a = integrate_args(cache, pr, slot_ids, rays_per_probe, env);
    if (a.probes == 0) return GI_OK;
    const unsigned blocks = (a.probes + kIntThreads / 4 - 1) / (kIntThreads / 4);
    if (rays_per_probe == 64) k_integrate<true><<<blocks, kIntThreads, 0, (cudaStream_t)stream>>>(a);
    else k_integrate<false><<<blocks, kIntThreads, 0, (cudaStream_t)stream>>>(a);
    return cuda_status(cudaGetLastError(), "k_integrate launch");
}

gi_status gi_probes_integrate_nrc(gi_cache_t cache, gi_nrc_t nrc, const gi_probes *pr, const uint32_t *slot_ids,
                                  uint32_t rays_per_probe, const float env[3], gi_stream_t stream) {
    gi_status s = integrate_check(cache, pr, slot_ids, rays_per_probe);
    if (s != GI_OK) return s;
    if (!nrc) {
        set_error("gi_probes_integrate_nrc: NULL surrogate");
        return GI_ERR_INVALID_ARG;
    }
    s = ensure_moments();
    if (s != GI_OK) return s;
    IntegrateArgs a = integrate_args(cache, pr, slot_ids, rays_per_probe, env);
    if (a.probes == 0) return GI_OK;
    const uint64_t n = (uint64_t)a.probes * rays_per_probe;
    s = nrc_override(nrc, n, &a.ovr_bits, &a.ovr);
    if (s != GI_OK) return s;
    const unsigned blocks = (a.probes + kIntThreads / 4 - 1) / (kIntThreads / 4);
    if (rays_per_probe == 64) k_integrate_surr<true><<<blocks, kIntThreads, 0, (cudaStream_t)stream>>>(a);
    else k_integrate_surr<false><<<blocks, kIntThreads, 0, (cudaStream_t)stream>>>(a);
    return cuda_status(cudaGetLastError(), "k_integrate_surr launch");
}

gi_status gi_probes_gather(gi_cache_t cache, const gi_probes *pr, const uint32_t *slot_ids, const float *ray_len,
                           uint32_t rays_per_probe, const float env[3], float *atlas, gi_stream_t stream) {
    gi_status s = integrate_check(cache, pr, slot_ids, rays_per_probe);
    if (s != GI_OK) return s;
    if ((!ray_len || !atlas) && pr->layout.num_probes > 0) {
        set_error("gi_probes_gather: NULL ray_len or atlas");
        return GI_ERR_INVALID_ARG;
    }
    if ((uintptr_t)atlas & 15) {
        set_error("gi_probes_gather: atlas must be 16-byte aligned");
        return GI_ERR_INVALID_ARG;
    }
    IntegrateArgs a = integrate_args(cache, pr, slot_ids, rays_per_probe, env);
    if (a.probes == 0) return GI_OK;
    a.ray_len = ray_len;
    k_gather<<<(a.probes + 7) / 8, 256, 0, (cudaStream_t)stream>>>(a, reinterpret_cast<float4 *>(atlas));
    return cuda_status(cudaGetLastError(), "k_gather launch");
}

gi_status gi_probes_filter(const gi_probes *pr, const gi_view *view, const float *atlas_in, float *atlas_out,
                           uint32_t axis, gi_stream_t stream) {
    if (!pr || !view_ok(view) || !pr->mask || !pr->pos || !pr->nrm || axis > 1 ||
        ((!atlas_in || !atlas_out) && pr->layout.num_probes > 0) || atlas_in == atlas_out) {
        set_error("gi_probes_filter: NULL argument, bad view or axis, or in-place atlas");
        return GI_ERR_INVALID_ARG;
    }
    if (((uintptr_t)atlas_in | (uintptr_t)atlas_out | (uintptr_t)pr->pos | (uintptr_t)pr->nrm) & 15) {
        set_error("gi_probes_filter: atlases and probe buffers must be 16-byte aligned");
        return GI_ERR_INVALID_ARG;
    }
    gi_status s = ensure_moments();
    if (s != GI_OK) return s;
    FilterArgs a;
    a.in = reinterpret_cast<const float4 *>(atlas_in);
    a.out = reinterpret_cast<float4 *>(atlas_out);
    a.mask = pr->mask;
    a.mi = mip_info(pr->layout);
    a.ppos = reinterpret_cast<const float4 *>(pr->pos);
    a.pnrm = reinterpret_cast<const float4 *>(pr->nrm);
    a.probes = pr->layout.num_probes;
    a.tiles_x = pr->layout.tiles_x;
    a.dscale = (float)distance_scale(view->fov_y, view->width, view->height);
    a.axis = (int)axis;
    if (a.probes == 0) return GI_OK;
    k_filter<<<(a.probes + kFiltProbes - 1) / kFiltProbes, 64 * kFiltProbes, 0, (cudaStream_t)stream>>>(a);
    return cuda_status(cudaGetLastError(), "k_filter launch");
}

gi_status gi_probes_project(const gi_probes *pr, const float *atlas, gi_stream_t stream) {
    if (!pr || !pr->nrm || !pr->sh || (!atlas && pr->layout.num_probes > 0) || ((uintptr_t)atlas & 15)) {
        set_error("gi_probes_project: NULL argument or misaligned atlas");
        return GI_ERR_INVALID_ARG;
    }
    gi_status s = ensure_moments();
    if (s != GI_OK) return s;
    const uint32_t P = pr->layout.num_probes;
    if (P == 0) return GI_OK;
    k_project<<<(P + kProjThreads / 4 - 1) / (kProjThreads / 4), kProjThreads, 0, (cudaStream_t)stream>>>(reinterpret_cast<const float4 *>(atlas),
                                                              reinterpret_cast<const float4 *>(pr->nrm), pr->sh, P);
    return cuda_status(cudaGetLastError(), "k_project launch");
}

gi_status gi_probes_interpolate(const gi_gbuffer *gbuf, const gi_view *view, const gi_probes *pr, float *out,
                                gi_stream_t stream) {
    gi_status s = interp_check(gbuf, view, pr, out);
    if (s != GI_OK) return s;
    const InterpArgs a = interp_args(gbuf, view, pr, out);
    dim3 grid(interp_grid_x(view->width), interp_grid_y(view->height));
    k_interpolate<<<grid, 256, 0, (cudaStream_t)stream>>>(a);
    return cuda_status(cudaGetLastError(), "k_interpolate launch");
}

} // extern "C"
