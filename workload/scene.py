"""Box scenes, camera paths, G-buffers and probe-ray hit records.

Recipe (all seeded; the seed of frame f of configuration c is
1234 + 1000*c + f):

* configuration 1 -- a Cornell box (floor, ceiling, back, left and right
  walls as thin boxes, two inner boxes, one emissive ceiling quad), albedo
  uniform in [0.2, 0.8] per channel, one point light under the ceiling,
  64x64 pixels, 60 degree vertical field of view, static camera, 256 rays per
  probe (4 per hemispherical cell);
* configuration 2 -- a 64 x 16 x 64 m room (6 walls) holding 4,090 random
  boxes with per-axis sizes log-uniform in [0.05, 5] m and centres uniform in
  the room; 2 % of the boxes are emissive with radiance uniform in [1, 50]
  per channel; 1920x1080 pixels, 64 rays per probe; the camera follows a
  closed Catmull-Rom spline through 8 seeded control points; one point light
  moves on a circle under the ceiling;
* configuration 4 -- the Cornell box of configuration 1 at 1920x1080, 64
  rays per probe, static camera, 128 frames (the learned-surrogate workload);
* configuration 5 -- the same recipe at 3840x2160 with 16,384 boxes in a
  96 x 20 x 96 m room, three of the emissive boxes moving on circles.

Hit radiance is direct light only: albedo/pi * sum_l I_l max(0, n.l) / r^2
(no shadow rays), plus the emission of emissive boxes, plus noise uniform in
[0, 0.05] per channel.  Rays that leave the scene return the environment
(zero) and are flagged by an infinite ray length.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_LIB_DIR, "libwltrace.so")

SEED_BASE = 1234
# record planes, in order, of the float32 array returned in Frame.records
REC_PLANES = ("px", "py", "pz", "nx", "ny", "nz", "r", "g", "b", "len", "dx", "dy", "dz")

CONFIGS = {
    1: dict(name="cornell-64x64", scene="cornell", width=64, height=64, fov_deg=60.0,
            rays_per_probe=256, log2_slots=16, cell_size=0.05, num_lods=4, alpha=0.1,
            evict_frames=8, frames=4, moving_camera=False, resolved_format=0),
    2: dict(name="boxes-1080p", scene="boxes", width=1920, height=1080, fov_deg=60.0,
            rays_per_probe=64, log2_slots=22, cell_size=0.05, num_lods=4, alpha=0.1,
            evict_frames=8, frames=64, moving_camera=True, n_boxes=4096,
            room=(64.0, 16.0, 64.0), moving_emitters=0, resolved_format=0, log2_tiles=18),
    5: dict(name="boxes-4k", scene="boxes", width=3840, height=2160, fov_deg=60.0,
            rays_per_probe=64, log2_slots=24, cell_size=0.05, num_lods=4, alpha=0.1,
            evict_frames=8, frames=64, moving_camera=True, n_boxes=16384,
            room=(96.0, 20.0, 96.0), moving_emitters=3, resolved_format=1, log2_tiles=20),
}
# The 1080p boxes workload at the paper's quarter-sample operating point: 2x2 temporal upscale (one
# probe per 16x16 spawn tile traces 64 rays), probes reprojected from the previous frame along the
# camera's motion vectors.
CONFIGS[6] = dict(CONFIGS[2], name="boxes-1080p-upscale2", upscale=2, motion=True)
# The paper's whole chain at that operating point: configuration 6 with the two-level world cache
# (8x8 tiles with MIP levels, 2^18 tile slots, min_samples 16) and the probe filter (Algorithm 5).
CONFIGS[7] = dict(CONFIGS[6], name="boxes-1080p-upscale2-tiles-filtered", tiles=True, min_samples=16,
                  filtered=True)


# Configuration 3: 16 independent views of uneven resolution, each its own seeded scene (Cornell
# boxes and small box rooms alternating), 64 rays per probe (0.23 M to 3.7 M records per view).
_VIEW_SIZES = ((640, 360), (1280, 720), (1920, 1080), (2560, 1440))


def batched_views(n_views: int = 16, sizes=_VIEW_SIZES):
    """Per-view configuration dicts of the batched workload (with their seed bases)."""
    views = []
    for v in range(n_views):
        w, h = sizes[v % len(sizes)]
        if v % 2 == 0:
            cfg = dict(CONFIGS[1], width=w, height=h, rays_per_probe=64, frames=32, moving_camera=False,
                       log2_slots=21 if w * h > 1_000_000 else 20)
        else:
            cfg = dict(CONFIGS[2], width=w, height=h, frames=32, n_boxes=512, room=(24.0, 8.0, 24.0),
                       log2_slots=21 if w * h > 1_000_000 else 20)
        cfg["name"] = f"view{v}-{cfg['scene']}-{w}x{h}"
        views.append((cfg, SEED_BASE + 3000 + 100 * v))
    return views


CONFIGS[3] = dict(name="batched-16-views", scene="batched", n_views=16, frames=32)

# Configuration 4: the Cornell box of configuration 1 seen at 1080p (static camera, 64 rays per
# probe), plus the learned surrogate: 16-level hash encoding with 2^19 entries per level and
# resolutions 16 .. 2048 over the box, trained on 65,536 resolved cells per frame (4 minibatches),
# queried for cold cells, dropped inserts and LOD >= 2; 128 frames.
CONFIGS[4] = dict(CONFIGS[1], name="cornell-1080p-surrogate", width=1920, height=1080, rays_per_probe=64,
                  log2_slots=20, frames=128, nrc_log2_table=19, nrc_batch=65536, nrc_train_steps=4,
                  nrc_query_lod=2, nrc_lr=2e-2, nrc_trust=0.05,
                  nrc_resolutions=(16, 22, 30, 42, 58, 80, 111, 153, 212, 294, 406, 561, 776, 1072, 1482, 2048))


# --------------------------------------------------------------------------- tracer
def build_tracer(force: bool = False) -> str:
    """Compile the C ray caster (gcc, OpenMP, no FP contraction)."""
    src = os.path.join(_HERE, "trace.c")
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(src):
        return _LIB_PATH
    os.makedirs(_LIB_DIR, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _tracer():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build_tracer())
        f = lib.wl_trace
        f.restype = ctypes.c_int
        f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                      ctypes.c_long, ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                      ctypes.c_int]
        _lib = lib
    return _lib


def trace(bmin, bmax, origins, dirs, tmax=1e30):
    """Closest hit of each ray: (t, box, face); t = inf and box = -1 on a miss."""
    bmin = np.ascontiguousarray(bmin, np.float32)
    bmax = np.ascontiguousarray(bmax, np.float32)
    o = np.ascontiguousarray(origins, np.float32).reshape(-1, 3)
    d = np.ascontiguousarray(dirs, np.float32).reshape(-1, 3)
    n = o.shape[0]
    t = np.empty(n, np.float32)
    box = np.empty(n, np.int32)
    face = np.empty(n, np.int32)
    rc = _tracer().wl_trace(bmin.ctypes.data, bmax.ctypes.data, bmin.shape[0], o.ctypes.data, d.ctypes.data,
                            n, tmax, t.ctypes.data, box.ctypes.data, face.ctypes.data,
                            max(1, os.cpu_count() or 1))
    if rc != 0:
        raise RuntimeError("wl_trace failed")
    return t, box, face


# --------------------------------------------------------------------------- scenes
@dataclass
class Scene:
    bmin: np.ndarray      # (nb, 3) float32
    bmax: np.ndarray      # (nb, 3) float32
    albedo: np.ndarray    # (nb, 3) float32
    emission: np.ndarray  # (nb, 3) float32
    moving: list = field(default_factory=list)  # [(box index, centre0, radius, phase)]
    kind: str = "boxes"
    room: tuple = (2.0, 2.0, 2.0)
    path: np.ndarray | None = None  # camera control points (8, 3) float64

    def at_frame(self, f: int, frames: int) -> "Scene":
        if not self.moving:
            return self
        bmin = self.bmin.copy()
        bmax = self.bmax.copy()
        for (b, c0, radius, phase) in self.moving:
            ang = 2.0 * math.pi * f / max(frames, 1) + phase
            c = np.array([c0[0] + radius * math.cos(ang), c0[1], c0[2] + radius * math.sin(ang)])
            half = 0.5 * (self.bmax[b].astype(np.float64) - self.bmin[b].astype(np.float64))
            bmin[b] = (c - half).astype(np.float32)
            bmax[b] = (c + half).astype(np.float32)
        return Scene(bmin, bmax, self.albedo, self.emission, self.moving, self.kind, self.room, self.path)


def _slab(lo, hi):
    return np.array(lo, np.float64), np.array(hi, np.float64)


def _cornell(rng: np.random.Generator) -> Scene:
    w = 0.05
    boxes = [
        _slab((-1 - w, -w, -1 - w), (1 + w, 0.0, 1 + w)),        # floor
        _slab((-1 - w, 2.0, -1 - w), (1 + w, 2.0 + w, 1 + w)),   # ceiling
        _slab((-1 - w, -w, -1 - w), (1 + w, 2.0 + w, -1.0)),     # back wall
        _slab((-1 - w, -w, -1 - w), (-1.0, 2.0 + w, 1 + w)),     # left wall
        _slab((1.0, -w, -1 - w), (1 + w, 2.0 + w, 1 + w)),       # right wall
    ]
    jit = rng.uniform(-0.1, 0.1, size=4)
    cs = np.array([-0.35 + jit[0], 0.0, 0.3 + jit[1]])
    ct = np.array([0.35 + jit[2], 0.0, -0.3 + jit[3]])
    boxes.append(_slab(cs + (-0.3, 0.0, -0.3), cs + (0.3, 0.6, 0.3)))   # short box
    boxes.append(_slab(ct + (-0.3, 0.0, -0.3), ct + (0.3, 1.2, 0.3)))   # tall box
    boxes.append(_slab((-0.25, 1.98, -0.25), (0.25, 2.0, 0.25)))        # emissive quad
    bmin = np.array([b[0] for b in boxes], np.float32)
    bmax = np.array([b[1] for b in boxes], np.float32)
    nb = len(boxes)
    albedo = rng.uniform(0.2, 0.8, size=(nb, 3)).astype(np.float32)
    emission = np.zeros((nb, 3), np.float32)
    emission[-1] = (10.0, 9.0, 7.5)
    return Scene(bmin, bmax, albedo, emission, [], "cornell", (2.0, 2.0, 2.0), None)


def _catmull_rom(p0, p1, p2, p3, t):
    t2, t3 = t * t, t * t * t
    return 0.5 * ((2.0 * p1) + (-p0 + p2) * t + (2.0 * p0 - 5.0 * p1 + 4.0 * p2 - p3) * t2
                  + (-p0 + 3.0 * p1 - 3.0 * p2 + p3) * t3)


def _path_point(path: np.ndarray, s: float) -> np.ndarray:
    n = path.shape[0]
    i = int(math.floor(s)) % n
    t = s - math.floor(s)
    return _catmull_rom(path[(i - 1) % n], path[i], path[(i + 1) % n], path[(i + 2) % n], t)


def _boxes(rng: np.random.Generator, cfg: dict) -> Scene:
    lx, ly, lz = cfg["room"]
    w = 0.2
    walls = [
        _slab((-w, -w, -w), (lx + w, 0.0, lz + w)),
        _slab((-w, ly, -w), (lx + w, ly + w, lz + w)),
        _slab((-w, -w, -w), (0.0, ly + w, lz + w)),
        _slab((lx, -w, -w), (lx + w, ly + w, lz + w)),
        _slab((-w, -w, -w), (lx + w, ly + w, 0.0)),
        _slab((-w, -w, lz), (lx + w, ly + w, lz + w)),
    ]
    # camera control points first, so that boxes can keep clear of the path
    path = np.stack([rng.uniform(0.15 * lx, 0.85 * lx, 8),
                     rng.uniform(1.5, min(8.0, 0.5 * ly), 8),
                     rng.uniform(0.15 * lz, 0.85 * lz, 8)], axis=1)
    samples = np.array([_path_point(path, 8.0 * k / 256.0) for k in range(256)])
    nrand = cfg["n_boxes"] - len(walls)
    lo_list, hi_list = [], []
    while len(lo_list) < nrand:
        c = rng.uniform((0.0, 0.0, 0.0), (lx, ly, lz))
        u = rng.uniform(0.0, 1.0, 3)
        size = np.array([0.05 * math.pow(100.0, float(x)) for x in u])
        lo, hi = c - 0.5 * size, c + 0.5 * size
        # keep a 0.5 m clearance around the camera path
        inside = np.all((samples > lo - 0.5) & (samples < hi + 0.5), axis=1)
        if inside.any():
            continue
        lo_list.append(lo)
        hi_list.append(hi)
    bmin = np.array([b[0] for b in walls] + lo_list, np.float32)
    bmax = np.array([b[1] for b in walls] + hi_list, np.float32)
    nb = bmin.shape[0]
    albedo = rng.uniform(0.2, 0.8, size=(nb, 3)).astype(np.float32)
    emissive = rng.uniform(0.0, 1.0, nb) < 0.02
    emissive[: len(walls)] = False
    emission = np.zeros((nb, 3), np.float32)
    emission[emissive] = rng.uniform(1.0, 50.0, size=(int(emissive.sum()), 3)).astype(np.float32)
    moving = []
    idx = np.nonzero(emissive)[0]
    for k in range(min(cfg.get("moving_emitters", 0), idx.size)):
        b = int(idx[k])
        c0 = 0.5 * (bmin[b].astype(np.float64) + bmax[b].astype(np.float64))
        moving.append((b, c0, float(rng.uniform(2.0, 6.0)), float(rng.uniform(0.0, 2.0 * math.pi))))
    return Scene(bmin, bmax, albedo, emission, moving, "boxes", (lx, ly, lz), path)


def make_scene(config, seed: int | None = None) -> Scene:
    """Scene of a configuration number (seeded by it) or of a configuration dict and seed."""
    cfg = CONFIGS[config] if isinstance(config, int) else config
    if seed is None:
        seed = SEED_BASE + 1000 * config
    rng = np.random.default_rng(seed)
    if cfg["scene"] == "cornell":
        return _cornell(rng)
    return _boxes(rng, cfg)


# --------------------------------------------------------------------------- camera
@dataclass
class Camera:
    pos: np.ndarray    # (3,) float32
    fwd: np.ndarray    # (3,) float32, unit
    right: np.ndarray  # (3,) float32, unit
    up: np.ndarray     # (3,) float32, unit
    fov_y: float       # radians
    width: int
    height: int


def _camera(scene: Scene, cfg: dict, f: int) -> Camera:
    if scene.kind == "cornell":
        pos = np.array([0.0, 1.0, 2.6])
        fwd = np.array([0.0, 0.0, -1.0])
    else:
        s = 1.0 * f / cfg["frames"]
        pos = _path_point(scene.path, s)
        ahead = _path_point(scene.path, s + 0.05)
        fwd = ahead - pos
        fwd[1] *= 0.3
        fwd /= np.linalg.norm(fwd)
    upw = np.array([0.0, 1.0, 0.0])
    right = np.cross(fwd, upw)
    right /= np.linalg.norm(right)
    up = np.cross(right, fwd)
    return Camera(pos.astype(np.float32), fwd.astype(np.float32), right.astype(np.float32),
                  up.astype(np.float32), math.radians(cfg["fov_deg"]), cfg["width"], cfg["height"])


def camera_rays(cam: Camera):
    """Unit directions (H, W, 3) float32 through the pixel centres.

    dir = fwd + sx*right + sy*up, sx = (2(x+0.5)/W - 1) tan(fov/2) W/H,
    sy = (1 - 2(y+0.5)/H) tan(fov/2); row 0 is the top of the image."""
    w, h = cam.width, cam.height
    th = np.float32(math.tan(0.5 * cam.fov_y))
    aspect = np.float32(w / h)
    xs = (np.float32(2.0) * (np.arange(w, dtype=np.float32) + np.float32(0.5)) / np.float32(w) - np.float32(1.0)) * th * aspect
    ys = (np.float32(1.0) - np.float32(2.0) * (np.arange(h, dtype=np.float32) + np.float32(0.5)) / np.float32(h)) * th
    d = (cam.fwd[None, None, :] + xs[None, :, None] * cam.right[None, None, :]
         + ys[:, None, None] * cam.up[None, None, :]).astype(np.float32)
    d /= np.sqrt((d * d).sum(axis=2, keepdims=True)).astype(np.float32)
    return d.astype(np.float32)


def _face_normals(face: np.ndarray) -> np.ndarray:
    n = np.zeros(face.shape + (3,), np.float32)
    ok = face >= 0
    ax = np.where(ok, face >> 1, 0)
    sgn = np.where((face & 1) == 1, 1.0, -1.0).astype(np.float32)
    for a in range(3):
        n[..., a] = np.where(ok & (ax == a), sgn, 0.0)
    return n


def render_gbuffer(scene: Scene, cam: Camera):
    """Returns (gbuffer (H, W, 4) float32 = (nx, ny, nz, distance), hit (H, W, 3))."""
    d = camera_rays(cam)
    o = np.broadcast_to(cam.pos, d.shape)
    t, box, face = trace(scene.bmin, scene.bmax, o, d)
    t = t.reshape(cam.height, cam.width)
    face = face.reshape(cam.height, cam.width)
    n = _face_normals(face)
    gb = np.empty((cam.height, cam.width, 4), np.float32)
    gb[..., :3] = n
    gb[..., 3] = t
    tt = np.where(np.isfinite(t), t, np.float32(0.0))
    hit = (cam.pos[None, None, :] + d * tt[..., None]).astype(np.float32)
    return gb, hit


# --------------------------------------------------------------------------- probes
def halton_jitter(frame: int, upscale: int = 1) -> tuple[int, int]:
    """(floor(8u H_2(frame+1)), floor(8u H_3(frame+1))) with exact integer digit reversal: the
    jitter inside a spawn tile of 8u x 8u pixels."""
    def fs(i: int, b: int) -> int:
        num, den = 0, 1
        while i > 0:
            i, dgt = divmod(i, b)
            num = num * b + dgt
            den *= b
        return (8 * upscale * num) // den
    return fs(frame + 1, 2), fs(frame + 1, 3)


def motion_vectors(gbuf: np.ndarray, cam: Camera, prev: Camera) -> np.ndarray:
    """Per pixel the offset (float32, pixels) from the pixel centre to the centre position of its
    surface point in the previous camera (static geometry); zero for sky pixels."""
    H, W = gbuf.shape[:2]
    d = camera_rays(cam).reshape(H, W, 3).astype(np.float64)
    dist = gbuf[..., 3].astype(np.float64)
    ok = np.isfinite(dist)
    X = cam.pos.astype(np.float64) + d * np.where(ok, dist, 0.0)[..., None]
    v = X - prev.pos.astype(np.float64)
    z = v @ prev.fwd.astype(np.float64)
    th = math.tan(0.5 * prev.fov_y)
    sx = (v @ prev.right.astype(np.float64)) / (z * th * prev.width / prev.height)
    sy = (v @ prev.up.astype(np.float64)) / (z * th)
    xp = (sx + 1.0) * 0.5 * prev.width
    yp = (1.0 - sy) * 0.5 * prev.height
    ys, xs = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    mv = np.zeros((H, W, 2), np.float32)
    good = ok & (z > 0)
    mv[..., 0] = np.where(good, xp - (xs + 0.5), 0.0)
    mv[..., 1] = np.where(good, yp - (ys + 0.5), 0.0)
    return mv


def _onb(n: np.ndarray):
    """Orthonormal basis around unit normals (Duff et al. 2017), float32."""
    one = np.float32(1.0)
    sign = np.where(np.signbit(n[..., 2]), np.float32(-1.0), one).astype(np.float32)
    a = (np.float32(-1.0) / (sign + n[..., 2])).astype(np.float32)
    b = (n[..., 0] * n[..., 1] * a).astype(np.float32)
    t = np.stack([one + sign * n[..., 0] * n[..., 0] * a, sign * b, -sign * n[..., 0]], axis=-1)
    bb = np.stack([b, sign + n[..., 1] * n[..., 1] * a, -n[..., 1]], axis=-1)
    return t.astype(np.float32), bb.astype(np.float32)


def _direct_light(scene: Scene, light_pos, light_I, pos, nrm, box):
    lvec = (light_pos[None, :] - pos).astype(np.float32)
    r2 = (lvec * lvec).sum(axis=1).astype(np.float32)
    r = np.sqrt(r2).astype(np.float32)
    cos = np.maximum((lvec * nrm).sum(axis=1) / np.maximum(r, np.float32(1e-6)), np.float32(0.0)).astype(np.float32)
    irr = (cos / np.maximum(r2, np.float32(1e-4))).astype(np.float32)
    alb = scene.albedo[box]
    rad = alb / np.float32(math.pi) * (irr[:, None] * light_I[None, :]) + scene.emission[box]
    return rad.astype(np.float32)


def _light(scene: Scene, f: int, frames: int):
    if scene.kind == "cornell":
        return np.array([0.0, 1.85, 0.0], np.float32), np.array([3.0, 3.0, 3.0], np.float32)
    lx, ly, lz = scene.room
    ang = 2.0 * math.pi * f / max(frames, 1)
    pos = np.array([0.5 * lx + 0.3 * lx * math.cos(ang), 0.75 * ly, 0.5 * lz + 0.3 * lz * math.sin(ang)])
    return pos.astype(np.float32), np.array([2000.0, 1800.0, 1600.0], np.float32)


@dataclass
class Frame:
    config: int
    frame: int
    camera: Camera
    gbuffer: np.ndarray      # (H, W, 4) float32: normal xyz, distance along the pixel ray (inf = sky)
    records: np.ndarray      # (13, R) float32 planes, see REC_PLANES
    rays_per_probe: int
    tiles_x: int
    tiles_y: int
    jitter: tuple
    probe_valid: np.ndarray  # (P,) bool: the tracer found a surface under the probe pixel
    light_pos: np.ndarray
    light_I: np.ndarray
    upscale: int = 1         # spawn tiles of 8u x 8u pixels: records belong to the spawn tiles
    spawn_x: int = 0         # spawn tiles per row / column (the tile grid when upscale is 1)
    spawn_y: int = 0
    motion: np.ndarray | None = None  # (H, W, 2) float32 motion vectors to the previous frame

    @property
    def n_records(self) -> int:
        return self.records.shape[1]


def make_frame(config, f: int, scene: Scene | None = None, rays_per_probe: int | None = None,
               seed_base: int | None = None, upscale: int | None = None, motion: bool | None = None) -> Frame:
    """Frame f of a configuration number or of a configuration dict (then seed_base is required;
    the frame's random draws use seed_base + f).  With upscale u one probe per spawn tile of
    8u x 8u pixels traces rays (records are spawn-tile major); with motion the frame carries the
    motion vectors to frame f - 1 (zero at f = 0)."""
    cfg = CONFIGS[config] if isinstance(config, int) else config
    if seed_base is None:
        seed_base = SEED_BASE + 1000 * config
    if scene is None:
        scene = make_scene(config, seed_base)
    upscale = cfg.get("upscale", 1) if upscale is None else upscale
    motion = cfg.get("motion", False) if motion is None else motion
    frames = cfg["frames"]
    sc = scene.at_frame(f, frames)
    cam = _camera(sc, cfg, f if cfg["moving_camera"] else 0)
    gb, hit = render_gbuffer(sc, cam)
    rng = np.random.default_rng(seed_base + f)
    rpp = rays_per_probe or cfg["rays_per_probe"]
    W, H = cam.width, cam.height
    tx_n, ty_n = (W + 7) // 8, (H + 7) // 8
    st = 8 * upscale
    sx_n, sy_n = (W + st - 1) // st, (H + st - 1) // st
    jx, jy = halton_jitter(f, upscale)
    tx, ty = np.meshgrid(np.arange(sx_n), np.arange(sy_n))
    px = np.minimum(st * tx + jx, W - 1).reshape(-1)
    py = np.minimum(st * ty + jy, H - 1).reshape(-1)
    P = px.size
    dist = gb[py, px, 3]
    valid = np.isfinite(dist)
    n = gb[py, px, :3]
    n_safe = np.where(valid[:, None], n, np.array([0.0, 0.0, 1.0], np.float32)).astype(np.float32)
    org = (hit[py, px] + n_safe * np.float32(1e-3)).astype(np.float32)
    t_ax, b_ax = _onb(n_safe)
    k = np.arange(rpp)
    cell = k & 63
    ci = (cell & 7).astype(np.float32)
    cj = (cell >> 3).astype(np.float32)
    ab = rng.random((P, rpp, 2), dtype=np.float32)
    u = np.float32(-1.0) + (ci[None, :] + ab[..., 0]) * np.float32(0.25)
    v = np.float32(-1.0) + (cj[None, :] + ab[..., 1]) * np.float32(0.25)
    x = (u + v) * np.float32(0.5)
    y = (u - v) * np.float32(0.5)
    z = np.float32(1.0) - np.abs(x) - np.abs(y)
    inv = np.float32(1.0) / np.sqrt(x * x + y * y + z * z)
    x, y, z = x * inv, y * inv, z * inv
    d = (x[..., None] * t_ax[:, None, :] + y[..., None] * b_ax[:, None, :] + z[..., None] * n_safe[:, None, :])
    d = (d / np.sqrt((d * d).sum(axis=2, keepdims=True))).astype(np.float32)
    o = np.broadcast_to(org[:, None, :], d.shape)
    t, box, face = trace(sc.bmin, sc.bmax, o.reshape(-1, 3), d.reshape(-1, 3))
    R = P * rpp
    d = d.reshape(R, 3)
    vrec = np.repeat(valid, rpp)
    hitm = np.isfinite(t) & vrec
    pos = np.zeros((R, 3), np.float32)
    pos[hitm] = (o.reshape(-1, 3)[hitm] + d[hitm] * t[hitm, None]).astype(np.float32)
    nrm = _face_normals(np.where(hitm, face, -1))
    lp, li = _light(sc, f, frames)
    rad = np.zeros((R, 3), np.float32)
    if hitm.any():
        rad[hitm] = _direct_light(sc, lp, li, pos[hitm], nrm[hitm], box[hitm])
    rad[hitm] += rng.uniform(0.0, 0.05, size=(int(hitm.sum()), 3)).astype(np.float32)
    ln = np.where(hitm, t, np.float32(np.inf)).astype(np.float32)
    ln[~vrec] = np.float32(-1.0)
    rec = np.empty((13, R), np.float32)
    rec[0:3] = pos.T
    rec[3:6] = nrm.T
    rec[6:9] = rad.T
    rec[9] = ln
    rec[10:13] = d.T
    mv = None
    if motion:
        prev_cam = _camera(scene.at_frame(max(f - 1, 0), frames), cfg, max(f - 1, 0) if cfg["moving_camera"] else 0)
        mv = motion_vectors(gb, cam, prev_cam)
    return Frame(config if isinstance(config, int) else -1, f, cam, gb, np.ascontiguousarray(rec), rpp, tx_n, ty_n,
                 (jx, jy), valid, lp, li, upscale, sx_n, sy_n, mv)


def make_frames(config: int, frames: int | None = None, start: int = 0, **kw):
    scene = make_scene(config)
    n = frames if frames is not None else CONFIGS[config]["frames"]
    return [make_frame(config, f, scene, **kw) for f in range(start, start + n)]


def records_random(n: int, seed: int, extent: float = 4.0, cam=(0.0, 0.0, 0.0), miss_frac: float = 0.05):
    """Unstructured records (13, n) for cache-only tests: positions uniform in a cube of side
    2*extent around the camera, axis-aligned or random unit normals, radiance in [0, 2)."""
    rng = np.random.default_rng(seed)
    rec = np.zeros((13, n), np.float32)
    rec[0:3] = (rng.uniform(-extent, extent, (3, n)) + np.asarray(cam, np.float64)[:, None]).astype(np.float32)
    nv = rng.normal(size=(3, n))
    nv /= np.linalg.norm(nv, axis=0, keepdims=True)
    rec[3:6] = nv.astype(np.float32)
    rec[6:9] = rng.uniform(0.0, 2.0, (3, n)).astype(np.float32)
    rec[9] = rng.uniform(0.0, 3.0, n).astype(np.float32)
    rec[9][rng.uniform(0, 1, n) < miss_frac] = np.float32(np.inf)
    dv = rng.normal(size=(3, n))
    dv /= np.linalg.norm(dv, axis=0, keepdims=True)
    rec[10:13] = dv.astype(np.float32)
    return rec
