"""Seeded synthetic inputs for the Gaussian Mesh Renderer workloads.

This module builds meshes, per-face attributes and pinhole cameras. It holds
none of the renderer's arithmetic (no conversion, projection or compositing):
both the FP64 oracle and the CUDA path consume what it produces, so that the
two sides see bit-identical FP32 inputs.

The paper optimises a unit sphere of about 40K facets against 253 hemisphere
views of dataset objects (Sec. 3.1). The datasets are not available, so
icospheres with analytic or procedural radial displacements, viewed from rings
and Fibonacci spheres of cameras, stand in for them.

Camera convention: world-to-camera rotation ``R`` (row-major 3x3) and
translation ``t`` (x_cam = R x_world + t), OpenCV axes (x right, y down,
z forward), pixel centres at integer + 0.5, principal point at the image
centre, focal length from a 50 degree field of view.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Packed camera record; field order and types match ``gmr_camera`` in the
# C ABI header: 16 float32, 2 int32, 1 float32; 76 bytes, no padding.
CAMERA_DTYPE = np.dtype(
    [
        ("R", np.float32, (9,)),
        ("t", np.float32, (3,)),
        ("fx", np.float32),
        ("fy", np.float32),
        ("cx", np.float32),
        ("cy", np.float32),
        ("width", np.int32),
        ("height", np.int32),
        ("znear", np.float32),
    ]
)

DEFAULT_FOV_DEG = 50.0
DEFAULT_ZNEAR = 0.01


# --------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------

def _icosahedron():
    """Regular icosahedron on the unit sphere.

    The 12 vertices are the cyclic permutations of (0, +-1, +-phi); the 20
    faces are found as the vertex triples whose three pairwise distances equal
    the edge length, oriented so that the normal points away from the origin.
    """
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    verts = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            verts.append((0.0, s1, s2 * phi))
            verts.append((s1, s2 * phi, 0.0))
            verts.append((s2 * phi, 0.0, s1))
    v = np.array(verts, dtype=np.float64)
    d2 = ((v[:, None, :] - v[None, :, :]) ** 2).sum(-1)
    edge2 = 4.0
    adj = np.abs(d2 - edge2) < 1e-9
    faces = []
    n = len(v)
    for i in range(n):
        for j in range(i + 1, n):
            if not adj[i, j]:
                continue
            for k in range(j + 1, n):
                if adj[i, k] and adj[j, k]:
                    a, b, c = v[i], v[j], v[k]
                    nrm = np.cross(b - a, c - a)
                    if np.dot(nrm, a + b + c) > 0:
                        faces.append((i, j, k))
                    else:
                        faces.append((i, k, j))
    f = np.array(faces, dtype=np.int64)
    assert f.shape == (20, 3)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v, f


def icosphere(level: int):
    """Icosphere of the given subdivision level on the unit sphere.

    Each level splits every triangle into four at its edge midpoints (one
    shared midpoint per edge), projected back onto the sphere, keeping the
    outward orientation. V = 10*4^L + 2, F = 20*4^L.
    Returns (vertices float64 [V,3], faces int32 [F,3]).
    """
    v, f = _icosahedron()
    for _ in range(level):
        nv = len(v)
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
        e_sorted = np.sort(e, axis=1)
        key = e_sorted[:, 0] * nv + e_sorted[:, 1]
        uniq, inv = np.unique(key, return_inverse=True)
        a = uniq // nv
        b = uniq % nv
        mid = v[a] + v[b]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        nf = len(f)
        m01 = nv + inv[0:nf]
        m12 = nv + inv[nf:2 * nf]
        m20 = nv + inv[2 * nf:3 * nf]
        f0, f1, f2 = f[:, 0], f[:, 1], f[:, 2]
        f = np.concatenate(
            [
                np.stack([f0, m01, m20], 1),
                np.stack([f1, m12, m01], 1),
                np.stack([f2, m20, m12], 1),
                np.stack([m01, m12, m20], 1),
            ],
            axis=0,
        )
        v = np.concatenate([v, mid], axis=0)
    return v, f.astype(np.int32)


def spherical_angles(v):
    """Polar angle from +z and azimuth atan2(y, x) of each row of ``v``."""
    r = np.linalg.norm(v, axis=1)
    theta = np.arccos(np.clip(v[:, 2] / r, -1.0, 1.0))
    phi = np.arctan2(v[:, 1], v[:, 0])
    return theta, phi


def radial_displace(v, radius):
    """Scale each unit-sphere vertex to the given radius (array or scalar)."""
    u = v / np.linalg.norm(v, axis=1, keepdims=True)
    return u * np.asarray(radius, dtype=np.float64).reshape(-1, 1)


def _fade(t):
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


def _smoothstep(t):
    return t * t * (3.0 - 2.0 * t)


def _perm_table(seed: int):
    rng = np.random.default_rng(seed)
    p = rng.permutation(256).astype(np.int64)
    return np.concatenate([p, p])


def perlin_noise3(points, seed: int):
    """Perlin's improved gradient noise (Perlin 2002) in [-1, 1] (approx.).

    Quintic fade, a seeded permutation of 0..255, and the twelve edge
    gradients of a cube selected by the low four hash bits.
    """
    perm = _perm_table(seed)
    p = np.asarray(points, dtype=np.float64)
    pi = np.floor(p).astype(np.int64)
    pf = p - pi
    X, Y, Z = (pi[:, 0] & 255), (pi[:, 1] & 255), (pi[:, 2] & 255)
    x, y, z = pf[:, 0], pf[:, 1], pf[:, 2]
    u, v, w = _fade(x), _fade(y), _fade(z)

    def grad(h, x, y, z):
        h = h & 15
        a = np.where(h < 8, x, y)
        b = np.where(h < 4, y, np.where((h == 12) | (h == 14), x, z))
        return np.where(h & 1, -a, a) + np.where(h & 2, -b, b)

    A = perm[X] + Y
    AA = perm[A] + Z
    AB = perm[A + 1] + Z
    B = perm[X + 1] + Y
    BA = perm[B] + Z
    BB = perm[B + 1] + Z

    def lerp(t, a, b):
        return a + t * (b - a)

    return lerp(
        w,
        lerp(v, lerp(u, grad(perm[AA], x, y, z), grad(perm[BA], x - 1, y, z)),
             lerp(u, grad(perm[AB], x, y - 1, z), grad(perm[BB], x - 1, y - 1, z))),
        lerp(v, lerp(u, grad(perm[AA + 1], x, y, z - 1), grad(perm[BA + 1], x - 1, y, z - 1)),
             lerp(u, grad(perm[AB + 1], x, y - 1, z - 1), grad(perm[BB + 1], x - 1, y - 1, z - 1))),
    )


def value_noise3(points, seed: int, freq: float = 4.0):
    """Seeded 3D value noise in [0, 1]: random lattice values at integer
    points of ``freq * p``, blended by smoothstep-weighted trilinear
    interpolation."""
    rng = np.random.default_rng(seed)
    table = rng.random(256)
    perm = _perm_table(seed + 7919)
    p = np.asarray(points, dtype=np.float64) * freq
    pi = np.floor(p).astype(np.int64)
    f = _smoothstep(p - pi)

    def val(ix, iy, iz):
        return table[perm[(perm[(perm[ix & 255] + iy) & 255] + iz) & 255]]

    x0, y0, z0 = pi[:, 0], pi[:, 1], pi[:, 2]
    out = np.zeros(len(p))
    for dx in (0, 1):
        wx = f[:, 0] if dx else 1.0 - f[:, 0]
        for dy in (0, 1):
            wy = f[:, 1] if dy else 1.0 - f[:, 1]
            for dz in (0, 1):
                wz = f[:, 2] if dz else 1.0 - f[:, 2]
                out += wx * wy * wz * val(x0 + dx, y0 + dy, z0 + dz)
    return out


# --------------------------------------------------------------------------
# cameras
# --------------------------------------------------------------------------

def look_at(position, width, height, fov_deg=DEFAULT_FOV_DEG, target=(0.0, 0.0, 0.0),
            up=(0.0, 0.0, 1.0), znear=DEFAULT_ZNEAR):
    """One pinhole camera at ``position`` looking at ``target`` (OpenCV axes).

    Rows of R are the camera's right, down and forward axes in world
    coordinates; t = -R * position. The focal length gives the stated field
    of view across the image width, and square pixels.
    """
    c = np.asarray(position, dtype=np.float64)
    fwd = np.asarray(target, dtype=np.float64) - c
    fwd /= np.linalg.norm(fwd)
    upv = np.asarray(up, dtype=np.float64)
    right = np.cross(fwd, upv)
    if np.linalg.norm(right) < 1e-6:
        right = np.cross(fwd, np.array([0.0, 1.0, 0.0]))
    right /= np.linalg.norm(right)
    down = np.cross(fwd, right)
    R = np.stack([right, down, fwd], 0)
    t = -R @ c
    cam = np.zeros((), dtype=CAMERA_DTYPE)
    cam["R"] = R.reshape(-1).astype(np.float32)
    cam["t"] = t.astype(np.float32)
    f = (width / 2.0) / math.tan(math.radians(fov_deg) / 2.0)
    cam["fx"] = f
    cam["fy"] = f
    cam["cx"] = width / 2.0
    cam["cy"] = height / 2.0
    cam["width"] = width
    cam["height"] = height
    cam["znear"] = znear
    return cam


def ring_cameras(n, elevation_deg, distance, width, height, azimuth0_deg=0.0):
    el = math.radians(elevation_deg)
    cams = np.zeros(n, dtype=CAMERA_DTYPE)
    for i in range(n):
        az = math.radians(azimuth0_deg) + 2.0 * math.pi * i / n
        pos = distance * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
        cams[i] = look_at(pos, width, height)
    return cams


def fibonacci_directions(n):
    """n nearly uniform unit vectors (golden-angle spiral)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ga = math.pi * (3.0 - math.sqrt(5.0))
    phi = ga * i
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], 1)


def fibonacci_cameras(n, distance, resolutions):
    """Cameras on a Fibonacci sphere; ``resolutions`` gives (W, H) per view."""
    d = fibonacci_directions(n)
    cams = np.zeros(n, dtype=CAMERA_DTYPE)
    for i in range(n):
        w, h = resolutions[i]
        cams[i] = look_at(distance * d[i], int(w), int(h))
    return cams


def random_view_cameras(rng, n, distance, width, height):
    d = rng.normal(size=(n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    cams = np.zeros(n, dtype=CAMERA_DTYPE)
    for i in range(n):
        cams[i] = look_at(distance * d[i], width, height)
    return cams


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

@dataclass
class Scene:
    """One synthetic problem: FP32 mesh, per-face attributes and cameras."""

    name: str
    verts: np.ndarray          # [V,3] float32
    faces: np.ndarray          # [F,3] int32
    rgb: np.ndarray            # [F,3] float32 (per-face colour)
    opacity: np.ndarray        # [F]   float32
    cams: np.ndarray           # [C]   CAMERA_DTYPE
    extra: dict = field(default_factory=dict)

    @property
    def n_pixels(self) -> int:
        return int(sum(int(c["width"]) * int(c["height"]) for c in self.cams))


def _seed(config: int, purpose: int) -> int:
    return config * 1000 + purpose


def scene_single_view(level=3, width=128, height=128):
    """Icosphere level 3 of radius 1, per-face RGB ~ U[0,1], opacity 0.9, one
    128x128 camera (fov 50) at distance 3; the target mesh has its vertices
    jittered by N(0, 0.02^2)."""
    v, f = icosphere(level)
    rng = np.random.default_rng(_seed(1, 1))
    rgb = rng.random((len(f), 3)).astype(np.float32)
    op = np.full(len(f), 0.9, dtype=np.float32)
    el, az = math.radians(20.0), math.radians(30.0)
    pos = 3.0 * np.array([math.cos(el) * math.cos(az), math.cos(el) * math.sin(az), math.sin(el)])
    cams = np.zeros(1, dtype=CAMERA_DTYPE)
    cams[0] = look_at(pos, width, height)
    jit = np.random.default_rng(_seed(1, 2)).normal(0.0, 0.02, size=v.shape)
    target_verts = (v + jit).astype(np.float32)
    return Scene("icosphere3_1x128", v.astype(np.float32), f, rgb, op, cams,
                 {"target_verts": target_verts})


def scene_ring(level=5, n_views=8, res=512):
    """Icosphere level 5 with r = 1 + 0.1 sin(4 theta) sin(3 phi), per-face
    RGB ~ U[0,1], opacity 0.9, 8 cameras on a ring at elevation 20 degrees,
    distance 3, 512x512. Target: same mesh with vertices jittered by
    N(0, 0.02^2)."""
    v, f = icosphere(level)
    th, ph = spherical_angles(v)
    v = radial_displace(v, 1.0 + 0.1 * np.sin(4 * th) * np.sin(3 * ph))
    rng = np.random.default_rng(_seed(2, 1))
    rgb = rng.random((len(f), 3)).astype(np.float32)
    op = np.full(len(f), 0.9, dtype=np.float32)
    cams = ring_cameras(n_views, 20.0, 3.0, res, res)
    jit = np.random.default_rng(_seed(2, 2)).normal(0.0, 0.02, size=v.shape)
    return Scene(f"icosphere{level}_sin_{n_views}x{res}", v.astype(np.float32), f, rgb, op, cams,
                 {"target_verts": (v + jit).astype(np.float32)})


RESOLUTION_SET = (256, 384, 512, 768, 1024)


def scene_fibonacci_uneven(level=6, n_views=64):
    """Icosphere level 6, r = 1, face RGB from seeded 3D value noise at the
    face centroids, 64 Fibonacci-sphere cameras at distance 3 with square
    resolutions drawn uniformly from {256,384,512,768,1024}."""
    v, f = icosphere(level)
    cen = v[f].mean(1)
    rgb = np.stack([value_noise3(cen, _seed(3, 10 + c)) for c in range(3)], 1).astype(np.float32)
    op = np.full(len(f), 0.9, dtype=np.float32)
    rng = np.random.default_rng(_seed(3, 1))
    res = rng.choice(RESOLUTION_SET, size=n_views)
    cams = fibonacci_cameras(n_views, 3.0, [(r, r) for r in res])
    jit = np.random.default_rng(_seed(3, 2)).normal(0.0, 0.02, size=v.shape)
    return Scene(f"icosphere{level}_noise_{n_views}xuneven", v.astype(np.float32), f, rgb, op, cams,
                 {"target_verts": (v + jit).astype(np.float32)})


def scene_large(level=8, n_views=16, res=1024):
    """Icosphere level 8 with seeded Perlin radial displacement of amplitude
    0.05 (noise sampled at 4x the unit-sphere point), per-face RGB ~ U[0,1],
    opacity 0.9, 16 Fibonacci cameras at distance 3, 1024x1024."""
    v, f = icosphere(level)
    n = perlin_noise3(4.0 * v + 0.5, _seed(4, 3))
    v = radial_displace(v, 1.0 + 0.05 * n)
    rng = np.random.default_rng(_seed(4, 1))
    rgb = rng.random((len(f), 3)).astype(np.float32)
    op = np.full(len(f), 0.9, dtype=np.float32)
    cams = fibonacci_cameras(n_views, 3.0, [(res, res)] * n_views)
    jit = np.random.default_rng(_seed(4, 2)).normal(0.0, 0.02, size=v.shape)
    return Scene(f"icosphere{level}_perlin_{n_views}x{res}", v.astype(np.float32), f, rgb, op, cams,
                 {"target_verts": (v + jit).astype(np.float32)})


def scene_fit(level=7, res=512, views_per_step=4, steps=200):
    """Optimisation-loop problem: a level-7 unit icosphere (face colours 0.5)
    fitted to renders of r = 1 + 0.15 sin(5 theta) cos(2 phi); each step
    draws 4 random views (uniform on the sphere, distance 3) at 512x512."""
    v, f = icosphere(level)
    th, ph = spherical_angles(v)
    target = radial_displace(v, 1.0 + 0.15 * np.sin(5 * th) * np.cos(2 * ph))
    rng = np.random.default_rng(_seed(5, 1))
    rgb_target = rng.random((len(f), 3)).astype(np.float32)
    rgb0 = np.full((len(f), 3), 0.5, dtype=np.float32)
    op = np.full(len(f), 0.9, dtype=np.float32)
    vrng = np.random.default_rng(_seed(5, 2))
    view_sets = [random_view_cameras(vrng, views_per_step, 3.0, res, res) for _ in range(steps)]
    return Scene(f"icosphere{level}_fit_{views_per_step}x{res}", v.astype(np.float32), f, rgb0, op,
                 view_sets[0], {"target_verts": target.astype(np.float32), "target_rgb": rgb_target,
                                "view_sets": view_sets})


def random_triangle_soup(seed, n_faces, spread=0.6, size=0.15, n_views=1, res=(64, 48)):
    """Small random scene: independent triangles around the origin, random
    colours and opacities in [0.2, 1], cameras on a ring. For edge cases
    (ragged image sizes, overlapping layers, varied shapes)."""
    rng = np.random.default_rng(seed)
    centers = rng.uniform(-spread, spread, size=(n_faces, 3))
    offs = rng.normal(0.0, size, size=(n_faces, 3, 3))
    v = (centers[:, None, :] + offs).reshape(-1, 3)
    f = np.arange(3 * n_faces, dtype=np.int32).reshape(-1, 3)
    rgb = rng.random((n_faces, 3)).astype(np.float32)
    op = rng.uniform(0.2, 1.0, size=n_faces).astype(np.float32)
    w, h = res
    cams = ring_cameras(n_views, 25.0, 3.0, w, h, azimuth0_deg=17.0)
    return Scene(f"soup{n_faces}", v.astype(np.float32), f, rgb, op, cams)


def scenes_by_name():
    return {
        "icosphere3_1x128": scene_single_view,
        "icosphere5_sin_8x512": scene_ring,
        "icosphere6_noise_64xuneven": scene_fibonacci_uneven,
        "icosphere8_perlin_16x1024": scene_large,
        "icosphere7_fit_4x512": scene_fit,
    }
