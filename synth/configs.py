"""Named synthetic workloads: camera rigs, scenes over time and method parameters.

Each workload mirrors the scale of one evaluation setting: image sizes,
number of input views, samples per ray, depth range and truncation.  The
geometry (where the planes and spheres are) is this module's choice; only
the counts and ranges come from the workload definitions.

Every input is seeded: textures by `tex_seed`, depth noise by a counter hash
of (seed, frame, view).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable

import numpy as np

from . import Camera, Scene, camera_at, look_at, render

DEPTH_NOISE_SIGMA = 0.002  # metres; makes the confidence weights non-trivial


def _rig_scene(frame: int, seed: int) -> Scene:
    """Static back wall, floor and side wall; one sphere moving +x at 1 cm/frame."""
    return Scene(
        planes=[(0.0, 0.0, 1.0, 6.0, 0.80, 0.72, 0.60),    # back wall z = 6
                (0.0, 1.0, 0.0, 1.2, 0.45, 0.60, 0.40),    # floor y = 1.2 (y down)
                (1.0, 0.0, 0.0, -2.0, 0.55, 0.55, 0.85)],  # side wall x = -2
        spheres=[(-0.15 + 0.01 * frame, 0.0, 2.0, 0.3, 0.90, 0.35, 0.25)],
        tex_seed=seed)


def _arc_scene(frame: int, seed: int) -> Scene:
    """Back plane z=1.5, floor y=0.8, left wall x=-1.2 and a sphere r=0.35."""
    return Scene(
        planes=[(0.0, 0.0, 1.0, 1.5, 0.80, 0.72, 0.60),
                (0.0, 1.0, 0.0, 0.8, 0.45, 0.60, 0.40),
                (1.0, 0.0, 0.0, -1.2, 0.55, 0.55, 0.85)],
        spheres=[(0.1, 0.0, 0.2, 0.35, 0.90, 0.35, 0.25)],
        tex_seed=seed)


def _three_sphere_scene(frame: int, seed: int) -> Scene:
    """Static walls plus three spheres with seeded velocities of 0.5-2 cm/frame, bouncing in a box."""
    rng = np.random.default_rng(seed + 1000)
    lo = np.array([-0.8, -0.5, 1.5])
    hi = np.array([0.8, 0.5, 3.5])
    spheres = []
    cols = [(0.90, 0.35, 0.25), (0.25, 0.80, 0.35), (0.30, 0.40, 0.90)]
    for s in range(3):
        p0 = rng.uniform(lo + 0.3, hi - 0.3)
        v = rng.normal(size=3)
        v = v / np.linalg.norm(v) * rng.uniform(0.005, 0.02)
        p = p0 + v * frame
        # reflect into [lo+0.25, hi-0.25]
        a, b = lo + 0.25, hi - 0.25
        span = b - a
        q = np.mod(p - a, 2 * span)
        p = a + np.where(q > span, 2 * span - q, q)
        spheres.append((p[0], p[1], p[2], 0.25) + cols[s])
    return Scene(planes=[(0.0, 0.0, 1.0, 8.0, 0.80, 0.72, 0.60),
                         (0.0, 1.0, 0.0, 1.2, 0.45, 0.60, 0.40),
                         (1.0, 0.0, 0.0, -2.5, 0.55, 0.55, 0.85)],
                 spheres=spheres, tex_seed=seed)


@dataclass
class Workload:
    name: str
    inputs: list
    targets: list            # per frame the same target list unless target_at is given
    num_samples: int
    z_near: float
    z_far: float
    mu: float
    tau: float = 0.03
    n_frames: int = 1
    seed: int = 0
    noise_sigma: float = DEPTH_NOISE_SIGMA
    scene_at: Callable[[int, int], Scene] = _rig_scene
    target_at: Callable[[int], list] | None = None
    notes: str = ""
    extra: dict = field(default_factory=dict)

    def scene(self, frame: int) -> Scene:
        return self.scene_at(frame, self.seed)

    def targets_at(self, frame: int) -> list:
        return self.target_at(frame) if self.target_at else self.targets

    def render_inputs(self, frame: int = 0, threads: int | None = None):
        """(rgba uint8 [N, H, W, 4], depth float32 [N, H, W]) of every input view at `frame`."""
        sc = self.scene(frame)
        rgbs, deps = [], []
        for k, cam in enumerate(self.inputs):
            rgb, dep = render(sc, cam, noise_seed=(self.seed * 1_000_003 + frame) & (2**63 - 1),
                              noise_sigma=self.noise_sigma, view_id=k, threads=threads)
            rgbs.append(rgb)
            deps.append(dep)
        return np.stack(rgbs), np.stack(deps)

    def render_target_gt(self, cam: Camera, frame: int = 0, threads: int | None = None):
        """Noise-free render of a target camera (ground truth colour and analytic depth)."""
        return render(self.scene(frame), cam, noise_sigma=0.0, threads=threads)


def rig_2x4(width, height, spacing=0.10):
    xs = [-1.5 * spacing, -0.5 * spacing, 0.5 * spacing, 1.5 * spacing]
    ys = [-0.5 * spacing, 0.5 * spacing]
    return [camera_at(width, height, (x, y, 0.0)) for y in ys for x in xs]


def rig_4x4(width, height, spacing=0.10):
    vs = [-1.5 * spacing, -0.5 * spacing, 0.5 * spacing, 1.5 * spacing]
    return [camera_at(width, height, (x, y, 0.0)) for y in vs for x in vs]


def arc_cameras(width, height, degrees, radius=2.0):
    cams = []
    for d in degrees:
        a = np.radians(d)
        cams.append(look_at(width, height, (radius * np.sin(a), 0.0, -radius * np.cos(a)), (0.0, 0.0, 0.0)))
    return cams


def plain_320x240(seed: int = 0) -> Workload:
    """4 inputs at 320x240 on a 30-degree arc of radius 2 m, target at the arc midpoint; D=64 on [0.5, 5], mu=0.05."""
    return Workload("plain_fp32_4x320x240_D64", arc_cameras(320, 240, [-15, -5, 5, 15]),
                    arc_cameras(320, 240, [0]), 64, 0.5, 5.0, 0.05, seed=seed, scene_at=_arc_scene)


def video_8x720p(seed: int = 0) -> Workload:
    """8 inputs at 1280x720 on a 2x4 rig (10 cm), 30 frames, one target moving inside the rig; D=128 on [0.3, 8]."""
    def tgt(frame):
        return [camera_at(1280, 720, (-0.15 + 0.3 * frame / 29.0, 0.0, 0.0))]
    return Workload("video_fp32_8x1280x720_D128", rig_2x4(1280, 720), tgt(0), 128, 0.3, 8.0, 0.04,
                    n_frames=30, seed=seed, scene_at=_rig_scene, target_at=tgt)


def diff_640x360(seed: int = 0) -> Workload:
    """Arc geometry at 640x360 with D=96 (the differentiable setting)."""
    return Workload("diff_fp32_4x640x360_D96", arc_cameras(640, 360, [-15, -5, 5, 15]),
                    arc_cameras(640, 360, [0]), 96, 0.5, 5.0, 0.05, seed=seed, scene_at=_arc_scene)


def batched_16_targets(seed: int = 0) -> Workload:
    """8 inputs at 1280x720; 16 targets of four sizes on a 4x4 grid; 2 frames."""
    sizes = [(640, 360), (960, 540), (1280, 720), (1920, 1080)]
    xs = np.linspace(-0.12, 0.12, 4)
    ys = np.linspace(-0.04, 0.04, 4)
    targets = []
    n = 0
    for y in ys:
        for x in xs:
            w, h = sizes[n % 4]
            targets.append(camera_at(w, h, (x, y, 0.0)))
            n += 1
    return Workload("batched_fp32_8x1280x720_16targets_D128", rig_2x4(1280, 720), targets, 128, 0.3, 8.0, 0.04,
                    n_frames=2, seed=seed, scene_at=_rig_scene)


def mixed_16x1080p(seed: int = 0) -> Workload:
    """16 inputs at 1920x1080 on a 4x4 rig; stereo targets (6.4 cm IPD); D=192 on [0.3, 10]; 120 frames."""
    return Workload("mixed_f16bf16_16x1920x1080_D192", rig_4x4(1920, 1080),
                    [camera_at(1920, 1080, (-0.032, 0.0, 0.0)), camera_at(1920, 1080, (0.032, 0.0, 0.0))],
                    192, 0.3, 10.0, 0.04, n_frames=120, seed=seed, scene_at=_three_sphere_scene)


def headline_8x1080p(seed: int = 0) -> Workload:
    """The 2x4 rig (10 cm) at 1920x1080, all 8 views fused into one 1920x1080 target inside the rig; D=128 on [0.3, 8]."""
    return Workload("fuse+splat_fp32_8x1920x1080_to_1920x1080_D128", rig_2x4(1920, 1080),
                    [camera_at(1920, 1080, (0.02, 0.01, 0.0))], 128, 0.3, 8.0, 0.04,
                    n_frames=30, seed=seed, scene_at=_rig_scene)


def tiny(width=48, height=32, n_views=3, num_samples=24, seed=0) -> Workload:
    """Small arc workload for fast oracle-vs-GPU checks (several tiles plus ragged tails)."""
    degs = np.linspace(-12, 12, n_views).tolist()
    return Workload(f"tiny_{n_views}x{width}x{height}_D{num_samples}", arc_cameras(width, height, degs),
                    arc_cameras(width, height, [1.5]), num_samples, 0.5, 5.0, 0.05, seed=seed, scene_at=_arc_scene)


ALL = {
    "plain": plain_320x240,
    "video": video_8x720p,
    "diff": diff_640x360,
    "batched": batched_16_targets,
    "mixed": mixed_16x1080p,
    "headline": headline_8x1080p,
}
