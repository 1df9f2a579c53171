"""Seeded synthetic 3DGS scenes.

This module only draws random splat sets with the shape of captured 3DGS
models; it holds none of the simplification arithmetic, so both the CUDA path
and the FP64 oracle can take their inputs from it.

Parameterisation (standard 3DGS, the input and output of Algorithm 1):
  xyz        (n, 3)  float32  centre mu
  log_scale  (n, 3)  float32  per-axis log of the standard deviation s
  rot        (n, 4)  float32  quaternion (w, x, y, z), not necessarily unit
  logit      (n,)    float32  opacity logit, alpha = sigmoid(logit)
  sh         (n, F)  float32  appearance feature f (F = 48 at SH degree 3:
                              3 DC values followed by 45 higher-band values)

Scene recipes (normal distributions are given as N(mean, standard deviation)):
  * surfaces_unit_cube: 8 surfaces in [0,1]^3, alternating spheres (centre
    U(0.25,0.75)^3, radius U(0.1,0.25)) and square planes (random normal,
    side U(0.3,0.7)); points uniform in area, equal count per surface, normal
    jitter N(0, 0.01).
  * patches_cube: n_patches surfaces in a 20 m cube, alternating spheres
    (radius U(0.5,2.5)) and square planes (side U(1,5)), centres U(2,18)^3;
    each patch gets a density multiplier log-uniform on [1,10] and a point
    count proportional to area x multiplier; normal jitter N(0, 0.01).
    Optionally a fraction of near-degenerate splats (one axis log-scale
    U(-12,-9)) and a fraction of duplicated centres (mu copied exactly from
    another random splat; all other attributes stay the splat's own).
  Attributes: log-scale N(-4.5, 0.5) per axis, rotation uniform on S^3
  (normalised 4-D Gaussian), opacity logit N(0, 1.5), SH DC N(0, 0.5), SH
  higher bands N(0, 0.05). The final splat order is a seeded random
  permutation, as in a densified 3DGS model whose order carries no locality.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SH_DIM = 48


@dataclasses.dataclass
class Scene:
    xyz: np.ndarray
    log_scale: np.ndarray
    rot: np.ndarray
    logit: np.ndarray
    sh: np.ndarray

    @property
    def n(self) -> int:
        return int(self.xyz.shape[0])

    def subset(self, idx) -> "Scene":
        return Scene(*(np.ascontiguousarray(a[idx]) for a in self.arrays()))

    def arrays(self):
        return (self.xyz, self.log_scale, self.rot, self.logit, self.sh)

    def copy(self) -> "Scene":
        return Scene(*(a.copy() for a in self.arrays()))

    @property
    def nbytes(self) -> int:
        return sum(a.nbytes for a in self.arrays())


def _attributes(rng: np.random.Generator, n: int, sh_dim: int = SH_DIM):
    log_scale = rng.normal(-4.5, 0.5, size=(n, 3)).astype(np.float32)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    rot = q.astype(np.float32)
    logit = rng.normal(0.0, 1.5, size=n).astype(np.float32)
    sh = np.empty((n, sh_dim), dtype=np.float32)
    ndc = min(3, sh_dim)
    sh[:, :ndc] = rng.normal(0.0, 0.5, size=(n, ndc))
    if sh_dim > ndc:
        sh[:, ndc:] = rng.normal(0.0, 0.05, size=(n, sh_dim - ndc))
    return log_scale, rot, logit, sh


def _orthonormal_frame(rng: np.random.Generator):
    nrm = rng.normal(size=3)
    nrm /= np.linalg.norm(nrm)
    a = np.array([1.0, 0.0, 0.0]) if abs(nrm[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(nrm, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(nrm, e1)
    return nrm, e1, e2


def _sphere_points(rng, centre, radius, m, jitter):
    d = rng.normal(size=(m, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius + rng.normal(0.0, jitter, size=(m, 1))
    return centre + d * r


def _plane_points(rng, centre, side, m, jitter):
    nrm, e1, e2 = _orthonormal_frame(rng)
    a = rng.uniform(-side / 2, side / 2, size=(m, 1))
    b = rng.uniform(-side / 2, side / 2, size=(m, 1))
    h = rng.normal(0.0, jitter, size=(m, 1))
    return centre + a * e1 + b * e2 + h * nrm


def _split_counts(weights: np.ndarray, n: int) -> np.ndarray:
    """Largest-remainder split of n into len(weights) integer counts."""
    w = weights / weights.sum()
    raw = w * n
    cnt = np.floor(raw).astype(np.int64)
    rest = n - int(cnt.sum())
    if rest > 0:
        order = np.argsort(-(raw - cnt), kind="stable")
        cnt[order[:rest]] += 1
    return cnt


def surfaces_unit_cube(n: int = 20000, seed: int = 0, n_surfaces: int = 8,
                       sh_dim: int = SH_DIM) -> Scene:
    """Small scene: n splats on 8 spheres/planes inside the unit cube."""
    rng = np.random.default_rng(seed)
    counts = _split_counts(np.ones(n_surfaces), n)
    pts = []
    for s in range(n_surfaces):
        if s % 2 == 0:
            c = rng.uniform(0.25, 0.75, size=3)
            pts.append(_sphere_points(rng, c, rng.uniform(0.1, 0.25), counts[s], 0.01))
        else:
            c = rng.uniform(0.25, 0.75, size=3)
            pts.append(_plane_points(rng, c, rng.uniform(0.3, 0.7), counts[s], 0.01))
    xyz = np.concatenate(pts).astype(np.float32)
    log_scale, rot, logit, sh = _attributes(rng, n, sh_dim)
    perm = rng.permutation(n)
    return Scene(np.ascontiguousarray(xyz[perm]), log_scale, rot, logit, sh)


def patches_cube(n: int, seed: int, n_patches: int = 64, cube: float = 20.0,
                 frac_degenerate: float = 0.0, frac_duplicate: float = 0.0,
                 sh_dim: int = SH_DIM) -> Scene:
    """Large scene: n splats on patches in a 20 m cube, density varying 10x."""
    rng = np.random.default_rng(seed)
    kinds = np.arange(n_patches) % 2  # 0 sphere, 1 plane
    radius = rng.uniform(0.5, 2.5, size=n_patches)
    side = rng.uniform(1.0, 5.0, size=n_patches)
    centres = rng.uniform(0.1 * cube, 0.9 * cube, size=(n_patches, 3))
    mult = np.exp(rng.uniform(0.0, math.log(10.0), size=n_patches))
    area = np.where(kinds == 0, 4.0 * math.pi * radius ** 2, side ** 2)
    counts = _split_counts(area * mult, n)
    pts = []
    for p in range(n_patches):
        if kinds[p] == 0:
            pts.append(_sphere_points(rng, centres[p], radius[p], counts[p], 0.01))
        else:
            pts.append(_plane_points(rng, centres[p], side[p], counts[p], 0.01))
    xyz = np.concatenate(pts).astype(np.float32)
    log_scale, rot, logit, sh = _attributes(rng, n, sh_dim)
    if frac_degenerate > 0:
        m = int(round(frac_degenerate * n))
        idx = rng.choice(n, size=m, replace=False)
        ax = rng.integers(0, 3, size=m)
        log_scale[idx, ax] = rng.uniform(-12.0, -9.0, size=m).astype(np.float32)
    if frac_duplicate > 0:
        m = int(round(frac_duplicate * n))
        dst = rng.choice(n, size=m, replace=False)
        src = rng.integers(0, n, size=m)
        xyz[dst] = xyz[src]
    perm = rng.permutation(n)
    return Scene(np.ascontiguousarray(xyz[perm]), log_scale[perm].copy(),
                 rot[perm].copy(), logit[perm].copy(), sh[perm].copy())


# Named workloads -----------------------------------------------------------

def workload(name: str) -> Scene:
    """The fixed, seeded scenes used by the tests and the benchmark."""
    if name == "unit20k":          # 20,000 splats, 8 surfaces, seed 0
        return surfaces_unit_cube(20000, seed=0)
    if name == "patches1m":        # 1,000,000 splats, 64 patches, seed 1
        return patches_cube(1_000_000, seed=1)
    if name == "patches6m":        # 6,000,000 splats, 5% degenerate, 1% duplicates
        return patches_cube(6_000_000, seed=2, frac_degenerate=0.05, frac_duplicate=0.01)
    if name == "patches200k":      # 200,000-splat precision-report scene, seed 3
        return patches_cube(200_000, seed=3, frac_degenerate=0.05, frac_duplicate=0.01)
    raise KeyError(name)



# Device-side generation ------------------------------------------------------
#
# The batched and serving workloads hold tens of millions of splats; drawing
# them with numpy takes about 1.7 s per million on one core.  These functions
# follow the patches_cube recipe above exactly (same distributions, same
# per-patch parameters, which are drawn on the host from default_rng(seed))
# but draw the per-splat values on the GPU with a torch generator seeded from
# the same seed, so the values differ from patches_cube(n, seed) while the
# distribution is the same.

def patches_cube_device(n: int, seed: int, device="cuda", n_patches: int = 64,
                        cube: float = 20.0, frac_degenerate: float = 0.0,
                        frac_duplicate: float = 0.0, sh_dim: int = SH_DIM):
    """patches_cube drawn on `device`; returns a tuple of 5 contiguous float32
    tensors (xyz, log_scale, rot, logit, sh)."""
    import torch
    rng = np.random.default_rng(seed)
    kinds = np.arange(n_patches) % 2
    radius = rng.uniform(0.5, 2.5, size=n_patches)
    side = rng.uniform(1.0, 5.0, size=n_patches)
    centres = rng.uniform(0.1 * cube, 0.9 * cube, size=(n_patches, 3))
    mult = np.exp(rng.uniform(0.0, math.log(10.0), size=n_patches))
    area = np.where(kinds == 0, 4.0 * math.pi * radius ** 2, side ** 2)
    counts = _split_counts(area * mult, n)
    frames = [_orthonormal_frame(rng) for _ in range(n_patches)]
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) * 7919 + 17)
    f32 = dict(dtype=torch.float32, device=device)
    pid = torch.repeat_interleave(torch.arange(n_patches, device=device),
                                  torch.as_tensor(counts, device=device))
    c = torch.as_tensor(centres, **f32)[pid]
    sph = torch.as_tensor(kinds == 0, device=device)[pid].unsqueeze(1)
    # spheres: direction on S^2 times radius + jitter
    d = torch.randn((n, 3), generator=g, **f32)
    d = d / d.norm(dim=1, keepdim=True)
    r = torch.as_tensor(radius, **f32)[pid].unsqueeze(1) + 0.01 * torch.randn((n, 1), generator=g, **f32)
    p_s = c + d * r
    # planes: uniform square in the patch frame + normal jitter
    nrm = torch.as_tensor(np.stack([f[0] for f in frames]), **f32)[pid]
    e1 = torch.as_tensor(np.stack([f[1] for f in frames]), **f32)[pid]
    e2 = torch.as_tensor(np.stack([f[2] for f in frames]), **f32)[pid]
    half = 0.5 * torch.as_tensor(side, **f32)[pid].unsqueeze(1)
    a = (torch.rand((n, 1), generator=g, **f32) * 2 - 1) * half
    b = (torch.rand((n, 1), generator=g, **f32) * 2 - 1) * half
    h = 0.01 * torch.randn((n, 1), generator=g, **f32)
    p_p = c + a * e1 + b * e2 + h * nrm
    xyz = torch.where(sph, p_s, p_p)
    del p_s, p_p, d, nrm, e1, e2
    log_scale = -4.5 + 0.5 * torch.randn((n, 3), generator=g, **f32)
    q = torch.randn((n, 4), generator=g, **f32)
    rot = q / q.norm(dim=1, keepdim=True)
    logit = 1.5 * torch.randn((n,), generator=g, **f32)
    sh = 0.05 * torch.randn((n, sh_dim), generator=g, **f32)
    ndc = min(3, sh_dim)
    sh[:, :ndc] *= 10.0  # DC: N(0, 0.5)
    if frac_degenerate > 0:
        m = int(round(frac_degenerate * n))
        idx = torch.randperm(n, generator=g, device=device)[:m]
        ax = torch.randint(0, 3, (m,), generator=g, device=device)
        log_scale[idx, ax] = -12.0 + 3.0 * torch.rand((m,), generator=g, **f32)
    if frac_duplicate > 0:
        m = int(round(frac_duplicate * n))
        dst = torch.randperm(n, generator=g, device=device)[:m]
        src = torch.randint(0, n, (m,), generator=g, device=device)
        xyz[dst] = xyz[src]
    perm = torch.randperm(n, generator=g, device=device)
    return tuple(t[perm].contiguous() for t in (xyz, log_scale, rot, logit, sh))


def batch_specs(n_scenes: int = 64, lo: int = 50_000, hi: int = 2_000_000,
                ratios=(0.5, 0.25, 0.1), seed: int = 1000):
    """Scene sizes (log-uniform on [lo, hi]), target ratios (uniform over
    `ratios`) and seeds (seed, seed+1, ...) of the batched workload."""
    rng = np.random.default_rng(seed - 1)
    sizes = np.exp(rng.uniform(math.log(lo), math.log(hi), n_scenes)).astype(np.int64)
    rs = np.asarray(ratios)[rng.integers(0, len(ratios), n_scenes)]
    return [(int(n), float(r), seed + i) for i, (n, r) in enumerate(zip(sizes, rs))]


def serve_specs(n_jobs: int = 200, rate: float = 20.0, lo: int = 20_000, hi: int = 6_000_000,
                ratios=(0.5, 0.1, 0.01), seed: int = 2000):
    """Poisson request stream: (arrival time s, size, ratio, scene seed) per
    job; sizes log-uniform on [lo, hi], ratios uniform over `ratios`."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate, n_jobs))
    t -= t[0]
    sizes = np.exp(rng.uniform(math.log(lo), math.log(hi), n_jobs)).astype(np.int64)
    rs = np.asarray(ratios)[rng.integers(0, len(ratios), n_jobs)]
    return [(float(a), int(n), float(r), seed + 1 + i)
            for i, (a, n, r) in enumerate(zip(t, sizes, rs))]
