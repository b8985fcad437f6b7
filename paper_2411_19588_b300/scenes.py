"""Seeded synthetic inputs for the underwater splat rasterizer.

This module only *draws* inputs: Gaussian parameter buffers, cameras and
water-medium vectors. It holds none of the rendering arithmetic (no
projection, compositing or medium model), so both the CUDA path and the FP64
oracle can be fed from it without sharing any of the method's code.

Workloads (sizes from the benchmark configurations):
  * ``tiny_scene``   -- 1,000 Gaussians in a box in front of one 128x96 camera
                        (fx=fy=120), SH degree 0, fixed medium.
  * ``patch_scene``  -- planar surface patches (Gaussians flattened along the
                        patch normal, minor log-scale -5) plus 10% floaters,
                        SH degree 3. Used at 300k Gaussians / 1280x854 and at
                        1.5M Gaussians / 1920x1280.
  * ``arc_cameras``  -- views on a 6 m arc around the scene centroid.

The paper evaluates on real underwater captures (Red Sea, Curacao, Panama and
its own TableDB, Sec. V-A); none of those is available here, and these
seeded scenes stand in for them with the same kind of structure: opaque
surfaces at 1-15 m seen through water with per-channel attenuation.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

# Real-SH degree-0 basis value 1/(2*sqrt(pi)); used here only to *encode* a
# drawn RGB colour into the DC coefficient, so that a degree-0 scene has the
# drawn colour as its view-independent colour.
_SH_DC = 0.5 / math.sqrt(math.pi)


@dataclasses.dataclass
class Camera:
    """Pinhole camera. Pixel (ix, iy) has its centre at (ix+0.5, iy+0.5);
    ``world_to_cam`` is a row-major 3x4 [R|t] with OpenCV axes (x right,
    y down, z forward)."""
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    world_to_cam: np.ndarray  # (3, 4) float64
    z_near: float = 0.2
    z_far: float = 20.0

    def as_array(self) -> np.ndarray:
        """Flat float64[20]: W, H, fx, fy, cx, cy, world_to_cam(12), z_near, z_far."""
        return np.concatenate([
            np.array([self.width, self.height, self.fx, self.fy, self.cx, self.cy], np.float64),
            np.asarray(self.world_to_cam, np.float64).reshape(12),
            np.array([self.z_near, self.z_far], np.float64)])

    @property
    def center(self) -> np.ndarray:
        R = np.asarray(self.world_to_cam, np.float64)[:, :3]
        t = np.asarray(self.world_to_cam, np.float64)[:, 3]
        return -R.T @ t


@dataclasses.dataclass
class Gaussians:
    """Structure-of-arrays Gaussian parameters (float32, C-contiguous)."""
    means: np.ndarray           # (n, 3)
    log_scales: np.ndarray      # (n, 3)
    quats: np.ndarray           # (n, 4) w, x, y, z; not necessarily unit
    opacity_logits: np.ndarray  # (n,)
    sh: np.ndarray              # (n, (deg+1)^2, 3)
    sh_degree: int

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def copy(self) -> "Gaussians":
        return Gaussians(self.means.copy(), self.log_scales.copy(), self.quats.copy(),
                         self.opacity_logits.copy(), self.sh.copy(), self.sh_degree)

    def subset(self, idx) -> "Gaussians":
        return Gaussians(np.ascontiguousarray(self.means[idx]), np.ascontiguousarray(self.log_scales[idx]),
                         np.ascontiguousarray(self.quats[idx]), np.ascontiguousarray(self.opacity_logits[idx]),
                         np.ascontiguousarray(self.sh[idx]), self.sh_degree)


@dataclasses.dataclass
class Medium:
    """Per-channel water parameters: attenuation beta_D, backscatter beta_B
    (both 1/m) and the veiling colour B_inf."""
    beta_d: np.ndarray
    beta_b: np.ndarray
    b_inf: np.ndarray

    def as_array(self) -> np.ndarray:
        """float32[9] = beta_D[3], beta_B[3], B_inf[3]."""
        return np.concatenate([self.beta_d, self.beta_b, self.b_inf]).astype(np.float32)


def look_at(eye, target, width, height, fx, fy, z_near=0.2, z_far=20.0) -> Camera:
    """Camera at ``eye`` looking at ``target`` with world -y as up."""
    eye = np.asarray(eye, np.float64)
    z = np.asarray(target, np.float64) - eye
    z /= np.linalg.norm(z)
    up = np.array([0.0, -1.0, 0.0])
    x = np.cross(z, up)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    t = -R @ eye
    w2c = np.concatenate([R, t[:, None]], axis=1)
    return Camera(width, height, float(fx), float(fy), width / 2.0, height / 2.0, w2c, z_near, z_far)


def _random_unit_quats(rng, n):
    q = rng.standard_normal((n, 4))
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _rotmat_to_quat(R):
    """Unit quaternions (w, x, y, z) of a stack of rotation matrices (Shepperd)."""
    R = np.asarray(R, np.float64)
    n = R.shape[0]
    q = np.empty((n, 4))
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    diag = np.stack([R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]], axis=1)
    case = np.where(tr > diag.max(axis=1), 3, diag.argmax(axis=1))
    m = case == 3
    s = np.sqrt(np.maximum(1.0 + tr[m], 1e-30)) * 2
    q[m, 0] = 0.25 * s
    q[m, 1] = (R[m, 2, 1] - R[m, 1, 2]) / s
    q[m, 2] = (R[m, 0, 2] - R[m, 2, 0]) / s
    q[m, 3] = (R[m, 1, 0] - R[m, 0, 1]) / s
    for i in range(3):
        m = case == i
        j, k = (i + 1) % 3, (i + 2) % 3
        s = np.sqrt(np.maximum(1.0 + R[m, i, i] - R[m, j, j] - R[m, k, k], 1e-30)) * 2
        q[m, 1 + i] = 0.25 * s
        q[m, 0] = (R[m, k, j] - R[m, j, k]) / s
        q[m, 1 + j] = (R[m, j, i] + R[m, i, j]) / s
        q[m, 1 + k] = (R[m, k, i] + R[m, i, k]) / s
    return q / np.linalg.norm(q, axis=1, keepdims=True)


def _sh_from_rgb(rng, n, rgb, degree, rest_std=0.1):
    k = (degree + 1) ** 2
    sh = np.zeros((n, k, 3), np.float64)
    sh[:, 0, :] = (rgb - 0.5) / _SH_DC
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, rest_std, (n, k - 1, 3))
    return sh


def tiny_scene(seed: int = 0):
    """1,000 Gaussians, means uniform in x,y in [-1,1] m, z in [1,6] m, in front
    of a 128x96 camera at the origin (fx=fy=120, centred principal point);
    log-scales ~N(-3,0.5), random unit quaternions, opacity logits ~N(0,1),
    SH degree 0 with RGB ~U[0,1]; medium beta_D=(0.40,0.20,0.10),
    beta_B=(0.30,0.25,0.20), B_inf=(0.05,0.20,0.30); far plane 20 m."""
    rng = np.random.default_rng(seed)
    n = 1000
    means = np.stack([rng.uniform(-1, 1, n), rng.uniform(-1, 1, n), rng.uniform(1, 6, n)], axis=1)
    log_scales = rng.normal(-3.0, 0.5, (n, 3))
    quats = _random_unit_quats(rng, n)
    logits = rng.normal(0.0, 1.0, n)
    rgb = rng.uniform(0, 1, (n, 3))
    sh = _sh_from_rgb(rng, n, rgb, 0)
    g = _as_gaussians(means, log_scales, quats, logits, sh, 0)
    medium = Medium(np.array([0.40, 0.20, 0.10], np.float32), np.array([0.30, 0.25, 0.20], np.float32),
                    np.array([0.05, 0.20, 0.30], np.float32))
    cam = Camera(128, 96, 120.0, 120.0, 64.0, 48.0, np.concatenate([np.eye(3), np.zeros((3, 1))], 1), 0.2, 20.0)
    return g, medium, cam


def random_medium(rng) -> Medium:
    """beta_D, beta_B ~ U[0.05, 0.6] per channel, B_inf ~ U[0.05, 0.4]."""
    return Medium(rng.uniform(0.05, 0.6, 3).astype(np.float32), rng.uniform(0.05, 0.6, 3).astype(np.float32),
                  rng.uniform(0.05, 0.4, 3).astype(np.float32))


def _as_gaussians(means, log_scales, quats, logits, sh, degree) -> Gaussians:
    f = lambda a: np.ascontiguousarray(a, dtype=np.float32)
    return Gaussians(f(means), f(log_scales), f(quats), f(logits), f(sh), degree)


def patch_scene(n: int, seed: int, z_range=(1.0, 8.0), width=1280, height=854, fx=1200.0,
                n_patches=40, floater_frac=0.10, sh_degree=3):
    """Surface-patch scene seen from a camera at the origin looking +z.

    ``n_patches`` square patches with centres at depth U[z_range] inside the
    frustum, side U[0.5,3] m and random normals with |n . view| >= 0.3. 90%
    of the Gaussians are spread uniformly (by area) over the patches, with
    tangent log-scale log(0.8*spacing)+N(0,0.2), normal log-scale -5, a
    random in-plane twist and opacity logit N(2,1). 10% are floaters uniform
    in the frustum volume with isotropic log-scale N(-3,0.5) and logit N(0,1).
    SH: DC colour U[0,1], other coefficients N(0,0.1). Returns
    (gaussians, medium, camera)."""
    rng = np.random.default_rng(seed)
    tanx, tany = 0.5 * width / fx, 0.5 * height / fx
    n_float = int(round(n * floater_frac))
    n_surf = n - n_float
    z0, z1 = z_range

    # patches
    pz = rng.uniform(z0, z1, n_patches)
    px = pz * rng.uniform(-0.8, 0.8, n_patches) * tanx
    py = pz * rng.uniform(-0.8, 0.8, n_patches) * tany
    centers = np.stack([px, py, pz], 1)
    views = centers / np.linalg.norm(centers, axis=1, keepdims=True)
    normals = np.empty((n_patches, 3))
    for i in range(n_patches):
        while True:
            v = rng.standard_normal(3)
            v /= np.linalg.norm(v)
            if abs(v @ views[i]) >= 0.3:
                break
        normals[i] = v if v @ views[i] < 0 else -v
    sides = rng.uniform(0.5, 3.0, n_patches)
    areas = sides ** 2
    owner = rng.choice(n_patches, size=n_surf, p=areas / areas.sum())
    counts = np.bincount(owner, minlength=n_patches)
    # tangent frames
    helper = np.where(np.abs(normals[:, :1]) < 0.9, np.array([[1.0, 0, 0]]), np.array([[0, 1.0, 0]]))
    t1 = np.cross(normals, helper)
    t1 /= np.linalg.norm(t1, axis=1, keepdims=True)
    t2 = np.cross(normals, t1)
    u = rng.uniform(-0.5, 0.5, n_surf) * sides[owner]
    v = rng.uniform(-0.5, 0.5, n_surf) * sides[owner]
    s_means = centers[owner] + u[:, None] * t1[owner] + v[:, None] * t2[owner]
    spacing = np.sqrt(areas / np.maximum(counts, 1))
    s_log = np.empty((n_surf, 3))
    s_log[:, 0] = np.log(0.8 * spacing[owner]) + rng.normal(0, 0.2, n_surf)
    s_log[:, 1] = np.log(0.8 * spacing[owner]) + rng.normal(0, 0.2, n_surf)
    s_log[:, 2] = -5.0
    twist = rng.uniform(0, 2 * np.pi, n_surf)
    c, s = np.cos(twist)[:, None], np.sin(twist)[:, None]
    e1 = c * t1[owner] + s * t2[owner]
    e2 = -s * t1[owner] + c * t2[owner]
    Rm = np.stack([e1, e2, normals[owner]], axis=2)  # columns: scale axes
    s_quats = _rotmat_to_quat(Rm)
    s_logits = rng.normal(2.0, 1.0, n_surf)

    # floaters: uniform in the frustum volume between z0 and z1
    zf = np.cbrt(rng.uniform(z0 ** 3, z1 ** 3, n_float))
    f_means = np.stack([zf * rng.uniform(-tanx, tanx, n_float), zf * rng.uniform(-tany, tany, n_float), zf], 1)
    f_log = np.repeat(rng.normal(-3.0, 0.5, (n_float, 1)), 3, axis=1)
    f_quats = _random_unit_quats(rng, n_float)
    f_logits = rng.normal(0.0, 1.0, n_float)

    means = np.concatenate([s_means, f_means])
    log_scales = np.concatenate([s_log, f_log])
    quats = np.concatenate([s_quats, f_quats])
    logits = np.concatenate([s_logits, f_logits])
    perm = rng.permutation(n)
    rgb = rng.uniform(0, 1, (n, 3))
    sh = _sh_from_rgb(rng, n, rgb, sh_degree)
    g = _as_gaussians(means[perm], log_scales[perm], quats[perm], logits[perm], sh, sh_degree)
    medium = random_medium(rng)
    cam = Camera(width, height, float(fx), float(fx), width / 2.0, height / 2.0,
                 np.concatenate([np.eye(3), np.zeros((3, 1))], 1), 0.2, 20.0)
    return g, medium, cam


def mid_scene(seed: int = 2, n: int = 300_000):
    """300k Gaussians at 1-8 m, 1280x854, fx=fy=1200, SH degree 3."""
    return patch_scene(n, seed, (1.0, 8.0), 1280, 854, 1200.0)


def full_scene(seed: int = 3, n: int = 1_500_000):
    """1.5M Gaussians at 2-15 m, 1920x1280, fx=fy=1800, SH degree 3."""
    return patch_scene(n, seed, (2.0, 15.0), 1920, 1280, 1800.0)


def arc_cameras(n_views: int, seed: int, centroid=(0.0, 0.0, 8.5), radius=8.5, arc_len=6.0,
                width=1920, height=1280, fx=1800.0, jitter=0.05):
    """``n_views`` cameras on an arc of length ``arc_len`` m and radius
    ``radius`` m about ``centroid`` (yaw spread arc_len/radius rad), each
    looking at the centroid with seeded jitter of the eye and target. The
    middle of the arc is the origin looking +z."""
    rng = np.random.default_rng(seed)
    spread = arc_len / radius
    yaws = np.linspace(-spread / 2, spread / 2, n_views) if n_views > 1 else np.zeros(1)
    c = np.asarray(centroid, np.float64)
    cams = []
    for yaw in yaws:
        eye = c + radius * np.array([-math.sin(yaw), 0.0, -math.cos(yaw)]) + rng.normal(0, jitter, 3)
        target = c + rng.normal(0, jitter, 3)
        cams.append(look_at(eye, target, width, height, fx, fx))
    return cams


def uneven_cameras(n_views: int, seed: int, **arc):
    """``n_views`` arc cameras with widths drawn from 640..1920 (multiples of
    32) and aspect ratios between 4:3 and 3:2; focal length scales with the
    width (fx = 0.9375 * width)."""
    rng = np.random.default_rng(seed)
    base = arc_cameras(n_views, seed + 1000, **arc)
    out = []
    for cam in base:
        w = int(rng.integers(20, 61)) * 32
        aspect = rng.uniform(4 / 3, 3 / 2)
        h = int(round(w / aspect))
        f = 0.9375 * w
        out.append(Camera(w, h, f, f, w / 2.0, h / 2.0, cam.world_to_cam.copy(), cam.z_near, cam.z_far))
    return out


def perturb(g: Gaussians, medium: Medium, seed: int = 1):
    """Perturbed copy: means N(0,0.02 m), log-scales N(0,0.1), opacity
    logits N(0,0.3), colour (DC) N(0,0.05), medium x(1+N(0,0.1))."""
    rng = np.random.default_rng(seed)
    p = g.copy()
    p.means += rng.normal(0, 0.02, p.means.shape).astype(np.float32)
    p.log_scales += rng.normal(0, 0.1, p.log_scales.shape).astype(np.float32)
    p.opacity_logits += rng.normal(0, 0.3, p.opacity_logits.shape).astype(np.float32)
    p.sh[:, 0, :] += (rng.normal(0, 0.05, (p.n, 3)) / _SH_DC).astype(np.float32)
    m = Medium(*(np.asarray(a * (1 + rng.normal(0, 0.1, 3)), np.float32) for a in (medium.beta_d, medium.beta_b, medium.b_inf)))
    return p, m


def mlp_init(seed: int):
    """Initial weights of the 3080 -> 128 -> 128 -> 9 warm-start MLP: He-normal
    hidden layers, output layer N(0, 0.01), zero hidden biases and output
    biases -0.957 (softplus -> 0.325, the centre of the beta range) and
    -1.237 (sigmoid -> 0.225, the centre of the B_inf range). FP32."""
    rng = np.random.default_rng(seed)
    f = lambda a: np.asarray(a, np.float32)
    return {"W1": f(rng.normal(0, math.sqrt(2.0 / 3080), (128, 3080))), "b1": f(np.zeros(128)),
            "W2": f(rng.normal(0, math.sqrt(2.0 / 128), (128, 128))), "b2": f(np.zeros(128)),
            "W3": f(rng.normal(0, 0.01, (9, 128))), "b3": f([-0.957] * 6 + [-1.237] * 3)}


def view_maps(seed: int, width: int, height: int, z_far: float = 20.0):
    """A synthetic rendered view for feature tests: image [3,H,W] with smooth
    gradients plus noise in [0, 1.2], depth [H,W] in (0, z_far] with a
    background region at exactly z_far and a few pixels on bin edges."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:height, 0:width]
    img = np.stack([0.5 + 0.4 * np.sin(xx / (7.0 + c) + yy / (11.0 - c)) for c in range(3)])
    img = np.clip(img + rng.normal(0, 0.1, img.shape), 0, 1.2).astype(np.float32)
    depth = rng.uniform(0.3, z_far, (height, width)).astype(np.float32)
    depth[: height // 4, : width // 3] = z_far
    edges = (np.arange(1, 8) * (z_far / 8.0)).astype(np.float32)
    depth.ravel()[rng.choice(depth.size, 7, replace=False)] = edges
    return img, depth


def _cross_t(a, b):
    """Row-wise cross product written out (torch.linalg's first call loads its
    libraries, tens of seconds on a fresh machine)."""
    import torch
    return torch.stack([a[:, 1] * b[:, 2] - a[:, 2] * b[:, 1], a[:, 2] * b[:, 0] - a[:, 0] * b[:, 2],
                        a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0]], 1)


def _rotmat_to_quat_t(R):
    """Torch version of _rotmat_to_quat (Shepperd), for device-side generation."""
    import torch
    tr = R[:, 0, 0] + R[:, 1, 1] + R[:, 2, 2]
    diag = torch.stack([R[:, 0, 0], R[:, 1, 1], R[:, 2, 2]], 1)
    dmax, darg = diag.max(1)
    case = torch.where(tr > dmax, torch.full_like(darg, 3), darg)
    q = torch.empty((R.shape[0], 4), dtype=R.dtype, device=R.device)
    m = case == 3
    s = torch.sqrt(torch.clamp(1.0 + tr[m], min=1e-30)) * 2
    q[m, 0] = 0.25 * s
    q[m, 1] = (R[m, 2, 1] - R[m, 1, 2]) / s
    q[m, 2] = (R[m, 0, 2] - R[m, 2, 0]) / s
    q[m, 3] = (R[m, 1, 0] - R[m, 0, 1]) / s
    for i in range(3):
        m = case == i
        j, k = (i + 1) % 3, (i + 2) % 3
        s = torch.sqrt(torch.clamp(1.0 + R[m, i, i] - R[m, j, j] - R[m, k, k], min=1e-30)) * 2
        q[m, 1 + i] = 0.25 * s
        q[m, 0] = (R[m, k, j] - R[m, j, k]) / s
        q[m, 1 + j] = (R[m, j, i] + R[m, i, j]) / s
        q[m, 1 + k] = (R[m, k, i] + R[m, i, k]) / s
    return q / q.norm(dim=1, keepdim=True)


def patch_scene_device(n: int, seed: int, z_range=(1.0, 8.0), width=1280, height=854, fx=1200.0, n_patches=40,
                       floater_frac=0.10, sh_degree=3, device="cuda"):
    """The patch_scene recipe drawn with torch's generator on the device (same
    distributions, different random stream), for generating many training
    scenes quickly. Returns the parameter dict of render.params_to_device."""
    import torch
    g = torch.Generator(device=device).manual_seed(int(seed))
    f64 = dict(device=device, dtype=torch.float64)

    def U(lo, hi, *shape):
        return lo + (hi - lo) * torch.rand(*shape, generator=g, **f64)

    def N(mu, sd, *shape):
        return mu + sd * torch.randn(*shape, generator=g, **f64)

    tanx, tany = 0.5 * width / fx, 0.5 * height / fx
    n_float = int(round(n * floater_frac))
    n_surf = n - n_float
    z0, z1 = z_range
    pz = U(z0, z1, n_patches)
    centers = torch.stack([pz * U(-0.8, 0.8, n_patches) * tanx, pz * U(-0.8, 0.8, n_patches) * tany, pz], 1)
    views = centers / centers.norm(dim=1, keepdim=True)
    # normals with |n . view| >= 0.3, facing the camera: first acceptable of 64 draws
    cand = N(0, 1, n_patches, 64, 3)
    cand = cand / cand.norm(dim=2, keepdim=True)
    dots = (cand * views[:, None, :]).sum(2)
    first = (dots.abs() >= 0.3).to(torch.int8).argmax(1)
    normals = cand[torch.arange(n_patches, device=device), first]
    normals = torch.where((normals * views).sum(1, keepdim=True) < 0, normals, -normals)
    sides = U(0.5, 3.0, n_patches)
    areas = sides ** 2
    owner = torch.multinomial(areas / areas.sum(), n_surf, replacement=True, generator=g)
    counts = torch.bincount(owner, minlength=n_patches).to(torch.float64)
    ex = torch.tensor([1.0, 0.0, 0.0], **f64).expand(n_patches, 3)
    ey = torch.tensor([0.0, 1.0, 0.0], **f64).expand(n_patches, 3)
    helper = torch.where(normals[:, :1].abs() < 0.9, ex, ey)
    t1 = _cross_t(normals, helper)
    t1 = t1 / t1.norm(dim=1, keepdim=True)
    t2 = _cross_t(normals, t1)
    u = U(-0.5, 0.5, n_surf) * sides[owner]
    v = U(-0.5, 0.5, n_surf) * sides[owner]
    s_means = centers[owner] + u[:, None] * t1[owner] + v[:, None] * t2[owner]
    spacing = torch.sqrt(areas / torch.clamp(counts, min=1))
    s_log = torch.empty((n_surf, 3), **f64)
    s_log[:, 0] = torch.log(0.8 * spacing[owner]) + N(0, 0.2, n_surf)
    s_log[:, 1] = torch.log(0.8 * spacing[owner]) + N(0, 0.2, n_surf)
    s_log[:, 2] = -5.0
    twist = U(0, 2 * math.pi, n_surf)
    c, s = torch.cos(twist)[:, None], torch.sin(twist)[:, None]
    e1 = c * t1[owner] + s * t2[owner]
    e2 = -s * t1[owner] + c * t2[owner]
    s_quats = _rotmat_to_quat_t(torch.stack([e1, e2, normals[owner]], 2))
    s_logits = N(2.0, 1.0, n_surf)
    zf = torch.pow(U(z0 ** 3, z1 ** 3, n_float), 1.0 / 3.0)
    f_means = torch.stack([zf * U(-tanx, tanx, n_float), zf * U(-tany, tany, n_float), zf], 1)
    f_log = N(-3.0, 0.5, n_float, 1).expand(n_float, 3)
    f_quats = N(0, 1, n_float, 4)
    f_quats = f_quats / f_quats.norm(dim=1, keepdim=True)
    f_logits = N(0.0, 1.0, n_float)
    perm = torch.randperm(n, generator=g, device=device)
    k = (sh_degree + 1) ** 2
    sh = torch.zeros((n, k, 3), **f64)
    sh[:, 0, :] = (U(0, 1, n, 3) - 0.5) / _SH_DC
    if k > 1:
        sh[:, 1:, :] = N(0, 0.1, n, k - 1, 3)
    f32 = lambda a: a.to(torch.float32).contiguous()
    return {"means": f32(torch.cat([s_means, f_means])[perm]), "log_scales": f32(torch.cat([s_log, f_log])[perm]),
            "quats": f32(torch.cat([s_quats, f_quats])[perm]),
            "opacity_logits": f32(torch.cat([s_logits, f_logits])[perm]), "sh": f32(sh), "sh_degree": sh_degree}


def water_view(seed: int, width: int, height: int, z_range=(1.5, 12.0), z_far: float = 20.0, shadow_frac: float = 0.03,
               shadow_block: int = 4):
    """Maps of one synthetic underwater view for the backscatter estimator:
    depth [H,W] (a seabed sloping from z_range[1] at the top to z_range[0]
    at the bottom, a few rocks standing closer, and open water at exactly
    z_far in the top corner), albedo [3,H,W] in [0.15, 1] (smooth colour
    fields plus texture), and a shadow mask [H,W] (bool; square blocks of
    shadow_block pixels covering about shadow_frac of the view, where the
    direct signal is absent). Also the drawn medium. The image itself is
    composed by the caller."""
    rng = np.random.default_rng(seed)
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)
    v = yy / max(1, height - 1)
    z0, z1 = z_range
    depth = z1 + (z0 - z1) * v
    for _ in range(6):
        cx, cy = rng.uniform(0, width), rng.uniform(0.3 * height, height)
        rad = rng.uniform(0.05, 0.15) * width
        bump = np.exp(-((xx - cx) ** 2 + (yy - cy) ** 2) / (2 * rad * rad))
        depth = depth - rng.uniform(0.2, 0.5) * (depth - z0 * 0.7) * bump
    depth[: height // 6, : width // 4] = z_far
    alb = np.stack([0.55 + 0.3 * np.sin(xx / rng.uniform(20, 60) + yy / rng.uniform(20, 60) + c) for c in range(3)])
    alb = np.clip(alb + rng.normal(0, 0.08, alb.shape), 0.15, 1.0)
    shadow = np.zeros((height, width), bool)
    bh, bw = max(1, height // shadow_block), max(1, width // shadow_block)
    n_blocks = max(1, int(round(shadow_frac * bh * bw)))
    picks = rng.choice(bh * bw, n_blocks, replace=False)
    for p in picks:
        by, bx = divmod(int(p), bw)
        shadow[by * shadow_block:(by + 1) * shadow_block, bx * shadow_block:(bx + 1) * shadow_block] = True
    return depth.astype(np.float32), alb.astype(np.float32), shadow, random_medium(rng)
