"""Seeded synthetic inputs: scenes, textures and batches of problems.

This module only builds input arrays (geometry, materials, lights, cameras and
parameter textures). It holds none of the method's arithmetic: no rendering,
no gradients, no variance estimation. Both the CUDA path and the FP64 oracle
consume what it returns, so it must stay free of either.

The paper's own scenes (the spiral of its teaser figure, the texture task of
its appendix figure) are not available, so these seeded procedural scenes
stand in for them with the same kind of structure: a spiral tube with
base-colour / metalness / roughness textures over a ground plane, a closed
box with an area light, and a noise-displaced sphere.

Scene dictionary layout (all float arrays float32, all int arrays int32):

  positions [nv,3], uvs [nv,2], tris [nt,3], tri_mat [nt], tri_light [nt]
  spheres [ns,8] = (cx, cy, cz, r, u0, u1, v0, v1), sph_mat [ns]
  mat_type [nm] (0 Lambert, 1 principled), mat_textured [nm], mat_const [nm,5]
  quads [nq,12] = (p0, e1, e2, Le): parallelogram area lights
  env [3], has_env, eye/target/up [3], fov_deg, width, height,
  tex_c, tex_h, tex_w, clamp_lo [C], clamp_hi [C], max_depth,
  spp_prop, spp_fd, seed, key_id
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

LAMBERT = 0
PRINCIPLED = 1

# parameter ranges: base colour / albedo, metalness, roughness
RANGE_BC = (0.0, 1.0)
RANGE_METAL = (0.0, 1.0)
RANGE_ROUGH = (0.05, 1.0)


@dataclass
class Workload:
    """One inverse-rendering problem: a scene, its initial and target textures."""
    name: str
    scene: dict
    init_tex: np.ndarray          # [H, W, C] float32
    target_tex: np.ndarray        # [H, W, C] float32
    extra: dict = field(default_factory=dict)


# --------------------------------------------------------------------------
# textures
# --------------------------------------------------------------------------

def value_noise(h: int, w: int, seed: int, octaves: int = 4, base: int = 4) -> np.ndarray:
    """Smooth value noise in [0, 1], shape [h, w]; octave o has a (base*2^o)^2 lattice."""
    rng = np.random.default_rng(seed)
    out = np.zeros((h, w), np.float64)
    amp, total = 1.0, 0.0
    ys = (np.arange(h) + 0.5) / h
    xs = (np.arange(w) + 0.5) / w
    for o in range(octaves):
        n = base * (2 ** o)
        lat = rng.random((n + 1, n + 1))
        gy, gx = ys * n, xs * n
        iy = np.minimum(gy.astype(np.int64), n - 1)
        ix = np.minimum(gx.astype(np.int64), n - 1)
        ty, tx = gy - iy, gx - ix
        sy = ty * ty * (3 - 2 * ty)
        sx = tx * tx * (3 - 2 * tx)
        a = lat[iy][:, ix]
        b = lat[iy][:, ix + 1]
        c = lat[iy + 1][:, ix]
        d = lat[iy + 1][:, ix + 1]
        top = a + (b - a) * sx[None, :]
        bot = c + (d - c) * sx[None, :]
        out += amp * (top + (bot - top) * sy[:, None])
        total += amp
        amp *= 0.5
    out /= total
    lo, hi = out.min(), out.max()
    return (out - lo) / max(hi - lo, 1e-12)


def principled_texture(h: int, w: int, seed: int) -> np.ndarray:
    """5-channel texture: base colour RGB in [0.05,0.95], metal in [0,1], roughness in [0.1,0.9]."""
    t = np.empty((h, w, 5), np.float32)
    for c in range(3):
        t[..., c] = 0.05 + 0.9 * value_noise(h, w, seed * 101 + c)
    t[..., 3] = value_noise(h, w, seed * 101 + 3)
    t[..., 4] = 0.1 + 0.8 * value_noise(h, w, seed * 101 + 4)
    return t


def uniform_texture(h: int, w: int, c: int, seed: int, lo: float = 0.1, hi: float = 0.9) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=(h, w, c)).astype(np.float32)


# --------------------------------------------------------------------------
# geometry helpers
# --------------------------------------------------------------------------

class _MeshBuilder:
    def __init__(self):
        self.pos, self.uv, self.tris, self.mat, self.light = [], [], [], [], []
        self.nv = 0

    def quad(self, p0, e1, e2, mat, light=-1, uv0=(0.0, 0.0), uv_size=(1.0, 1.0)):
        """Parallelogram p0, p0+e1, p0+e1+e2, p0+e2 as two triangles (normal along e1 x e2)."""
        p0, e1, e2 = (np.asarray(x, np.float64) for x in (p0, e1, e2))
        corners = [p0, p0 + e1, p0 + e1 + e2, p0 + e2]
        uvs = [(0, 0), (1, 0), (1, 1), (0, 1)]
        base = self.nv
        for c, (s, t) in zip(corners, uvs):
            self.pos.append(c)
            self.uv.append((uv0[0] + s * uv_size[0], uv0[1] + t * uv_size[1]))
        self.nv += 4
        self.tris += [(base, base + 1, base + 2), (base, base + 2, base + 3)]
        self.mat += [mat, mat]
        self.light += [light, light]

    def grid(self, pos: np.ndarray, uv: np.ndarray, mat: int):
        """pos [n+1, m+1, 3], uv [n+1, m+1, 2] -> 2*n*m triangles."""
        n, m = pos.shape[0] - 1, pos.shape[1] - 1
        base = self.nv
        self.pos.extend(pos.reshape(-1, 3))
        self.uv.extend(uv.reshape(-1, 2))
        self.nv += (n + 1) * (m + 1)
        idx = base + np.arange((n + 1) * (m + 1)).reshape(n + 1, m + 1)
        a, b = idx[:-1, :-1], idx[:-1, 1:]
        c, d = idx[1:, :-1], idx[1:, 1:]
        t1 = np.stack([a, c, d], -1).reshape(-1, 3)
        t2 = np.stack([a, d, b], -1).reshape(-1, 3)
        tris = np.stack([t1, t2], 1).reshape(-1, 3)
        self.tris.extend(tris.tolist())
        self.mat += [mat] * len(tris)
        self.light += [-1] * len(tris)

    def arrays(self):
        return dict(
            positions=np.asarray(self.pos, np.float32).reshape(-1, 3),
            uvs=np.asarray(self.uv, np.float32).reshape(-1, 2),
            tris=np.asarray(self.tris, np.int32).reshape(-1, 3),
            tri_mat=np.asarray(self.mat, np.int32),
            tri_light=np.asarray(self.light, np.int32),
        )


def _scene(mesh: dict, *, spheres=None, sph_mat=None, mat_type, mat_textured, mat_const,
           quads=None, env=None, eye, target, up=(0, 1, 0), fov_deg, width, height,
           tex_c, tex_h, tex_w, max_depth, spp_prop=1, spp_fd=1, seed=7, key_id=0):
    C = tex_c
    lo = np.array([RANGE_BC[0]] * 3 + [RANGE_METAL[0], RANGE_ROUGH[0]], np.float32)[:C]
    hi = np.array([RANGE_BC[1]] * 3 + [RANGE_METAL[1], RANGE_ROUGH[1]], np.float32)[:C]
    s = dict(mesh)
    s["spheres"] = np.asarray(spheres if spheres is not None else np.zeros((0, 8)), np.float32).reshape(-1, 8)
    s["sph_mat"] = np.asarray(sph_mat if sph_mat is not None else [], np.int32)
    s["mat_type"] = np.asarray(mat_type, np.int32)
    s["mat_textured"] = np.asarray(mat_textured, np.int32)
    s["mat_const"] = np.asarray(mat_const, np.float32).reshape(-1, 5)
    s["quads"] = np.asarray(quads if quads is not None else np.zeros((0, 12)), np.float32).reshape(-1, 12)
    s["has_env"] = int(env is not None)
    s["env"] = np.asarray(env if env is not None else (0, 0, 0), np.float32)
    s["eye"] = np.asarray(eye, np.float32)
    s["target"] = np.asarray(target, np.float32)
    s["up"] = np.asarray(up, np.float32)
    s["fov_deg"] = float(fov_deg)
    s["width"], s["height"] = int(width), int(height)
    s["tex_c"], s["tex_h"], s["tex_w"] = int(C), int(tex_h), int(tex_w)
    s["clamp_lo"], s["clamp_hi"] = lo, hi
    s["max_depth"] = int(max_depth)
    s["spp_prop"], s["spp_fd"] = int(spp_prop), int(spp_fd)
    s["seed"], s["key_id"] = int(seed), int(key_id)
    return s


def _light_quad(center, size, le, y_down=True):
    """Axis-aligned horizontal quad light facing -y (down) by default."""
    cx, cy, cz = center
    h = size / 2
    if y_down:   # e1 = +x, e2 = +z: e1 x e2 = -y
        p0, e1, e2 = (cx - h, cy, cz - h), (size, 0, 0), (0, 0, size)
    else:
        p0, e1, e2 = (cx - h, cy, cz - h), (0, 0, size), (size, 0, 0)
    return p0, e1, e2, le


def _quad_row(p0, e1, e2, le):
    return list(p0) + list(e1) + list(e2) + list(le)


# --------------------------------------------------------------------------
# scenes
# --------------------------------------------------------------------------

def box_scene(width=64, height=64, tex=32, max_depth=3, seed=7, key_id=0, spp_prop=1, spp_fd=1):
    """Closed box [-1,1]^3 of six textured Lambert quads, a textured sphere and a ceiling light.

    The 6 walls and the sphere map into tiles of a 4x2 atlas of one RGB albedo texture.
    """
    mb = _MeshBuilder()
    tile = (0.25, 0.5)
    walls = [  # inward-facing: e1 x e2 points into the box
        ((-1, -1, -1), (2, 0, 0), (0, 2, 0)),    # back  z=-1, normal +z
        ((-1, -1, 1), (0, 2, 0), (2, 0, 0)),     # front z=+1, normal -z
        ((-1, -1, -1), (0, 2, 0), (0, 0, 2)),    # left  x=-1, normal +x
        ((1, -1, -1), (0, 0, 2), (0, 2, 0)),     # right x=+1, normal -x
        ((-1, -1, -1), (0, 0, 2), (2, 0, 0)),    # floor y=-1, normal +y
        ((-1, 1, -1), (2, 0, 0), (0, 0, 2)),     # ceil  y=+1, normal -y
    ]
    for i, (p0, e1, e2) in enumerate(walls):
        mb.quad(p0, e1, e2, mat=0, uv0=((i % 4) * tile[0], (i // 4) * tile[1]), uv_size=tile)
    p0, e1, e2, le = _light_quad((0.0, 0.999, 0.0), 0.5, (10.0, 10.0, 10.0))
    mb.quad(p0, e1, e2, mat=1, light=0)
    quads = [_quad_row(p0, e1, e2, le)]
    spheres = [(0.3, -0.6, 0.0, 0.4, 0.5, 0.75, 0.5, 1.0)]  # tile 6 of the atlas
    s = _scene(mb.arrays(), spheres=spheres, sph_mat=[0],
               mat_type=[LAMBERT, LAMBERT], mat_textured=[1, 0],
               mat_const=[[0.5] * 5, [0.0] * 5], quads=quads, env=None,
               eye=(0, 0, 0.9), target=(0, 0, -1), fov_deg=60, width=width, height=height,
               tex_c=3, tex_h=tex, tex_w=tex, max_depth=max_depth,
               spp_prop=spp_prop, spp_fd=spp_fd, seed=seed, key_id=key_id)
    return s


def spiral_scene(width=256, height=256, segments=256, sides=16, tex=256, max_depth=5,
                 spp_prop=2, spp_fd=1, seed=7, key_id=0, turns=2.5):
    """Planar Archimedean spiral lifted into a helix, swept by a circle, over a 10x10 ground quad.

    The tube carries a textured principled material (base colour, metalness, roughness);
    the ground is a constant grey Lambert. Lights: constant environment (1) and one
    1x1 quad light (10) above the spiral. Camera 45 degrees above the horizon.
    """
    mb = _MeshBuilder()
    mb.quad((-5, 0, 5), (10, 0, 0), (0, 0, -10), mat=1)          # ground, normal +y
    s_ = np.linspace(0.0, 1.0, segments + 1)
    th = s_ * turns * 2 * math.pi
    R = 0.3 + 1.2 * s_
    cen = np.stack([R * np.cos(th), 0.35 + 0.5 * s_, R * np.sin(th)], -1)
    tan = np.gradient(cen, axis=0)
    tan /= np.linalg.norm(tan, axis=1, keepdims=True)
    up = np.array([0.0, 1.0, 0.0])
    B = np.cross(tan, up)
    B /= np.linalg.norm(B, axis=1, keepdims=True)
    N = np.cross(B, tan)
    phi = np.linspace(0.0, 2 * math.pi, sides + 1)
    r_tube = 0.15
    pos = cen[:, None, :] + r_tube * (np.cos(phi)[None, :, None] * N[:, None, :]
                                      + np.sin(phi)[None, :, None] * B[:, None, :])
    uv = np.stack(np.meshgrid(s_, phi / (2 * math.pi), indexing="ij"), -1)
    mb.grid(pos, uv, mat=0)
    p0, e1, e2, le = _light_quad((0.0, 4.0, 0.0), 1.0, (10.0, 10.0, 10.0))
    mb.quad(p0, e1, e2, mat=2, light=0)
    quads = [_quad_row(p0, e1, e2, le)]
    d = 5.0
    eye = (0.0, d * math.sin(math.pi / 4), d * math.cos(math.pi / 4))
    return _scene(mb.arrays(), mat_type=[PRINCIPLED, LAMBERT, LAMBERT], mat_textured=[1, 0, 0],
                  mat_const=[[0.5] * 5, [0.5, 0.5, 0.5, 0, 1], [0.0] * 5], quads=quads,
                  env=(1.0, 1.0, 1.0), eye=eye, target=(0, 0.4, 0), fov_deg=45,
                  width=width, height=height, tex_c=5, tex_h=tex, tex_w=tex,
                  max_depth=max_depth, spp_prop=spp_prop, spp_fd=spp_fd, seed=seed, key_id=key_id)


def displaced_sphere_scene(width=1024, height=1024, n_lat=320, n_lon=320, tex=2048, max_depth=8,
                           spp_prop=4, spp_fd=4, n_lights=4, amp=0.05, seed=7, key_id=0, noise_seed=5):
    """UV sphere (n_lat x n_lon x 2 triangles) displaced by 3-octave value noise, on a ground quad."""
    mb = _MeshBuilder()
    mb.quad((-6, 0, 6), (12, 0, 0), (0, 0, -12), mat=1)
    v = np.linspace(0.0, 1.0, n_lat + 1)
    u = np.linspace(0.0, 1.0, n_lon + 1)
    th = v * math.pi
    ph = u * 2 * math.pi
    n = np.stack([np.sin(th)[:, None] * np.cos(ph)[None, :],
                  np.cos(th)[:, None] * np.ones_like(ph)[None, :],
                  np.sin(th)[:, None] * np.sin(ph)[None, :]], -1)
    disp = value_noise(n_lat + 1, n_lon + 1, noise_seed, octaves=3)
    disp[:, -1] = disp[:, 0]                   # close the seam
    disp[0, :] = disp[0, 0]
    disp[-1, :] = disp[-1, 0]                  # single value at each pole
    r = 1.0 + amp * (2 * disp - 1)
    pos = n * r[..., None] + np.array([0.0, 1.1, 0.0])
    uv = np.stack(np.meshgrid(v, u, indexing="ij"), -1)[..., ::-1]
    mb.grid(pos, uv, mat=0)
    quads = []
    for k in range(n_lights):
        a = 2 * math.pi * k / max(n_lights, 1)
        p0, e1, e2, le = _light_quad((3.0 * math.cos(a), 4.0, 3.0 * math.sin(a)), 0.8, (8.0, 8.0, 8.0))
        mb.quad(p0, e1, e2, mat=2, light=k)
        quads.append(_quad_row(p0, e1, e2, le))
    eye = (0.0, 3.2, 4.2)
    return _scene(mb.arrays(), mat_type=[PRINCIPLED, LAMBERT, LAMBERT], mat_textured=[1, 0, 0],
                  mat_const=[[0.5] * 5, [0.5, 0.5, 0.5, 0, 1], [0.0] * 5], quads=quads,
                  env=(0.8, 0.8, 0.8), eye=eye, target=(0, 1.0, 0), fov_deg=40,
                  width=width, height=height, tex_c=5, tex_h=tex, tex_w=tex,
                  max_depth=max_depth, spp_prop=spp_prop, spp_fd=spp_fd, seed=seed, key_id=key_id)


# ---- small scenes with closed-form answers --------------------------------

def plane_scene(width=16, height=16, tex=8, env=(0.7, 0.8, 0.9), max_depth=2, principled=False,
                seed=3, key_id=0):
    """One large textured quad (y=0, normal +y) under a constant environment, seen from above."""
    mb = _MeshBuilder()
    mb.quad((-0.6, 0, 0.6), (1.2, 0, 0), (0, 0, -1.2), mat=0, uv0=(0.0, 0.0), uv_size=(1.0, 1.0))
    C = 5 if principled else 3
    return _scene(mb.arrays(), mat_type=[PRINCIPLED if principled else LAMBERT], mat_textured=[1],
                  mat_const=[[0.5] * 5], env=env, eye=(0.0, 1.0, 0.0), target=(0.0, 0.0, -0.001),
                  up=(0, 0, -1), fov_deg=50, width=width, height=height, tex_c=C, tex_h=tex, tex_w=tex,
                  max_depth=max_depth, seed=seed, key_id=key_id)


def furnace_scene(width=16, height=16, albedo=1.0, env=(1.0, 1.0, 1.0), max_depth=4, textured=False,
                  tex=8, seed=3, key_id=0):
    """Convex analytic sphere with a constant Lambert albedo in a constant environment."""
    mb = _MeshBuilder()
    mesh = mb.arrays()
    return _scene(mesh, spheres=[(0, 0, 0, 1.0, 0, 1, 0, 1)], sph_mat=[0],
                  mat_type=[LAMBERT], mat_textured=[int(textured)], mat_const=[[albedo] * 5],
                  env=env, eye=(0, 0, 4.0), target=(0, 0, 0), fov_deg=35,
                  width=width, height=height, tex_c=3, tex_h=tex, tex_w=tex,
                  max_depth=max_depth, seed=seed, key_id=key_id)


def emitting_box_scene(width=8, height=8, albedo=0.5, le=1.0, max_depth=3, seed=3, key_id=0):
    """Closed box [-1,1]^3 whose six inward-facing walls each emit Le and reflect with albedo."""
    mb = _MeshBuilder()
    walls = [((-1, -1, -1), (2, 0, 0), (0, 2, 0)), ((-1, -1, 1), (0, 2, 0), (2, 0, 0)),
             ((-1, -1, -1), (0, 2, 0), (0, 0, 2)), ((1, -1, -1), (0, 0, 2), (0, 2, 0)),
             ((-1, -1, -1), (0, 0, 2), (2, 0, 0)), ((-1, 1, -1), (2, 0, 0), (0, 0, 2))]
    quads = []
    for i, (p0, e1, e2) in enumerate(walls):
        mb.quad(p0, e1, e2, mat=0, light=i)
        quads.append(_quad_row(p0, e1, e2, (le, le, le)))
    return _scene(mb.arrays(), mat_type=[LAMBERT], mat_textured=[0], mat_const=[[albedo] * 5],
                  quads=quads, env=None, eye=(0.1, 0.05, 0.5), target=(-0.2, -0.1, -1), fov_deg=70,
                  width=width, height=height, tex_c=3, tex_h=4, tex_w=4, max_depth=max_depth,
                  seed=seed, key_id=key_id)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def workload_box(width=64, height=64, tex=32, max_depth=3, seed=7, key_id=0):
    """64x64 box + sphere, 32x32 RGB albedo, init U[0.1,0.9] (seed 1), target seed 2."""
    s = box_scene(width, height, tex, max_depth, seed=seed, key_id=key_id)
    return Workload("box64", s, uniform_texture(tex, tex, 3, 1), uniform_texture(tex, tex, 3, 2))


def workload_spiral(width=256, height=256, segments=256, sides=16, tex=256, max_depth=5,
                    spp_prop=2, spp_fd=1, seed=7, key_id=0, name=None):
    """Spiral tube over a ground quad; 5-channel principled textures from value noise (init 11, target 12)."""
    s = spiral_scene(width, height, segments, sides, tex, max_depth, spp_prop, spp_fd, seed, key_id)
    nm = name or f"spiral{width}_{2 * segments * sides}tri_tex{tex}"
    return Workload(nm, s, principled_texture(tex, tex, 11), principled_texture(tex, tex, 12))


def workload_sphere(width=1024, height=1024, n=320, tex=2048, max_depth=8, spp_prop=4, spp_fd=4,
                    seed=7, key_id=0, n_lights=4, name=None):
    s = displaced_sphere_scene(width, height, n, n, tex, max_depth, spp_prop, spp_fd, n_lights,
                               seed=seed, key_id=key_id)
    nm = name or f"dsphere{width}_{2 * n * n}tri_tex{tex}"
    return Workload(nm, s, principled_texture(tex, tex, 11), principled_texture(tex, tex, 12))


def workload_batch(n_problems=64, seed=4, scale=1.0):
    """Independent problems of uneven sizes: images {64..512}^2, 1k-50k triangles, textures 64^2-512^2 x5,
    depths 3..8, 1 FD + 2 proportional spp each. `scale` < 1 shrinks images (for tests)."""
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n_problems):
        img = int(rng.choice([64, 128, 256, 512]))
        img = max(8, int(img * scale))
        tex = int(rng.choice([64, 128, 256, 512]))
        depth = int(rng.integers(3, 9))
        tris = int(rng.integers(1000, 50001))
        if rng.random() < 0.5:
            sides = 16
            segs = max(8, tris // (2 * sides))
            w = workload_spiral(img, img, segs, sides, tex, depth, 2, 1, seed=100 + q, key_id=q,
                                name=f"p{q}_spiral")
        else:
            n = max(8, int(math.sqrt(tris / 2)))
            w = workload_sphere(img, img, n, tex, depth, 2, 1, seed=100 + q, key_id=q, n_lights=2,
                                name=f"p{q}_dsphere")
        out.append(w)
    return out


def _blobs(n, rng, k, emit_scale, dens_scale):
    """Sum of k Gaussian blobs of emission (RGB) and density on an n^3 grid (voxel centres)."""
    c = (np.arange(n, dtype=np.float32) + 0.5) / n * 2.0 - 1.0
    out = np.zeros((n, n, n, 4), np.float32)
    for _ in range(k):
        mu = rng.uniform(-0.55, 0.55, 3).astype(np.float32)
        s = np.float32(rng.uniform(0.12, 0.3))
        col = rng.uniform(0.2, 1.0, 3).astype(np.float32) * emit_scale
        rho = np.float32(rng.uniform(0.5, 1.0) * dens_scale)
        gx = np.exp(-((c - mu[0]) ** 2) / (2 * s * s))
        gy = np.exp(-((c - mu[1]) ** 2) / (2 * s * s))
        gz = np.exp(-((c - mu[2]) ** 2) / (2 * s * s))
        g = gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
        out[..., :3] += g[..., None] * col
        out[..., 3] += g * rho
    return out


def volume_scene(n=256, views=4, width=256, height=256, step=None, seed=7, key_id=0, bg=(0.0, 0.0, 0.0)):
    """An n^3 voxel volume in the box [-1, 1]^3 seen from `views` pinhole cameras on a circle of
    radius 3.2 around it (30 degrees above the equator), fov 40; march step one voxel (2/n)."""
    cams = []
    for v in range(views):
        a = 2.0 * math.pi * v / views
        eye = [3.2 * math.cos(a) * math.cos(0.5236), 3.2 * math.sin(0.5236), 3.2 * math.sin(a) * math.cos(0.5236)]
        cams.append(eye + [0.0, 0.0, 0.0] + [0.0, 1.0, 0.0] + [40.0])
    return {"kind": "volume", "nx": n, "ny": n, "nz": n, "lo": [-1.0, -1.0, -1.0], "hi": [1.0, 1.0, 1.0],
            "n_views": views, "width": width, "height": height, "cameras": np.asarray(cams, np.float32),
            "step": float(2.0 / n if step is None else step), "bg": list(bg), "seed": seed, "key_id": key_id,
            "clamp_lo": [0.0, 0.0, 0.0, 0.0], "clamp_hi": [4.0, 4.0, 4.0, 60.0]}


def workload_volume(n=256, views=4, width=256, height=256, seed=7, key_id=0):
    """Emissive-absorptive volume (the 256^3 x 4 = 67M-parameter experiment): target = eight
    Gaussian blobs of emission and density (seed 21), init = a uniform faint grey volume."""
    s = volume_scene(n, views, width, height, seed=seed, key_id=key_id)
    target = _blobs(n, np.random.default_rng(21), 8, 1.0, 12.0)
    init = np.empty((n, n, n, 4), np.float32)
    init[..., :3] = 0.2
    init[..., 3] = 1.0
    return Workload(f"volume{n}_{views}x{width}", s, init, target)

