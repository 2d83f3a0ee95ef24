"""Seeded synthetic RGB-D inputs: cameras, analytic scenes and their renders.

This module is an input generator shared by the FP64 oracle tests and the
CUDA path.  It holds none of the method's arithmetic.  The paper's inputs are
captured multi-camera video with fixed COLMAP poses and RAFT-Stereo depth
(Sec. 3, "Method"); the scenes here stand in for those captures at the same
image scales, with exact (optionally noised) z-depth from an FP64 ray caster.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "scene.c")
_OUT = os.path.join(_HERE, "_build", "libsynth.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the ray caster with gcc into synth/_build/libsynth.so."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            dp = ctypes.POINTER(ctypes.c_double)
            lib.synth_render.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp, ctypes.c_int,
                                         ctypes.c_uint64, ctypes.c_double, ctypes.c_int,
                                         ctypes.c_uint64, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_void_p]
            lib.synth_render.restype = ctypes.c_int
            _lib = lib
    return _lib


@dataclass
class Camera:
    """Pinhole camera; world->camera x_c = R x_w + t (OpenCV axes, y down, z forward).

    Pixel (i, j) has its centre at integer coordinates (column i, row j).
    """
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray = field(default_factory=lambda: np.eye(3))
    t: np.ndarray = field(default_factory=lambda: np.zeros(3))

    def pack(self) -> np.ndarray:
        return np.concatenate([[self.fx, self.fy, self.cx, self.cy],
                               np.asarray(self.R, np.float64).reshape(9),
                               np.asarray(self.t, np.float64).reshape(3)]).astype(np.float64)

    @property
    def centre(self) -> np.ndarray:
        return -np.asarray(self.R).T @ np.asarray(self.t)


def intrinsics(width: int, height: int, hfov_deg: float = 60.0):
    """Square pixels, principal point at the image centre, given horizontal FOV."""
    fx = (width / 2.0) / np.tan(np.radians(hfov_deg) / 2.0)
    return fx, fx, (width - 1) / 2.0, (height - 1) / 2.0


def camera_at(width, height, centre, R=None, hfov_deg=60.0) -> Camera:
    fx, fy, cx, cy = intrinsics(width, height, hfov_deg)
    R = np.eye(3) if R is None else np.asarray(R, np.float64)
    C = np.asarray(centre, np.float64)
    return Camera(width, height, fx, fy, cx, cy, R, -R @ C)


def look_at(width, height, centre, target, up=(0.0, -1.0, 0.0), hfov_deg=60.0) -> Camera:
    """Camera at `centre` whose +z axis points at `target` (y down)."""
    C = np.asarray(centre, np.float64)
    z = np.asarray(target, np.float64) - C
    z /= np.linalg.norm(z)
    x = np.cross(np.asarray(up, np.float64), z)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])  # rows: camera axes in world coordinates
    return camera_at(width, height, C, R, hfov_deg)


@dataclass
class Scene:
    """Planes (n.x = c) and spheres, each with a base RGB colour in [0, 1]."""
    planes: list = field(default_factory=list)   # (nx, ny, nz, c, r, g, b)
    spheres: list = field(default_factory=list)  # (px, py, pz, radius, r, g, b)
    tex_seed: int = 0
    tex_freq: float = 4.0
    octaves: int = 4


def render(scene: Scene, cam: Camera, noise_seed: int = 0, noise_sigma: float = 0.0,
           view_id: int = 0, threads: int | None = None):
    """Ray-cast one camera. Returns (rgba uint8 [H, W, 4], depth float32 [H, W])."""
    lib = _load()
    H, W = cam.height, cam.width
    rgba = np.empty((H, W, 4), np.uint8)
    depth = np.empty((H, W), np.float32)
    pc = np.ascontiguousarray(cam.pack())
    pl = np.ascontiguousarray(np.asarray(scene.planes, np.float64).reshape(-1, 7))
    sp = np.ascontiguousarray(np.asarray(scene.spheres, np.float64).reshape(-1, 7))
    dp = ctypes.POINTER(ctypes.c_double)
    if threads is None:
        threads = min(32, os.cpu_count() or 1)
    rc = lib.synth_render(pc.ctypes.data_as(dp), W, H,
                          pl.ctypes.data_as(dp), pl.shape[0], sp.ctypes.data_as(dp), sp.shape[0],
                          int(scene.tex_seed) & (2**64 - 1), float(scene.tex_freq), int(scene.octaves),
                          int(noise_seed) & (2**64 - 1), float(noise_sigma), int(view_id), int(threads),
                          rgba.ctypes.data, depth.ctypes.data)
    if rc != 0:
        raise ValueError("synth_render rejected its arguments")
    return rgba, depth


def rgba_to_u32(rgba: np.ndarray) -> np.ndarray:
    """View an [..., 4] uint8 RGBA array as packed little-endian uint32 words."""
    a = np.ascontiguousarray(rgba)
    return a.view(np.uint32).reshape(a.shape[:-1])
