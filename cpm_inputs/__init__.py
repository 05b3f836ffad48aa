"""Seeded synthetic inputs for the CPM hot path (shapes, interior boundaries,
boundary data, right-hand sides).

This module holds NO arithmetic of the method itself: it only describes
geometry and draws random data from fixed seeds.  Both the CUDA library's
tests/benchmark and the CPU oracle take their inputs from here, and neither
imports the other.

Workloads follow the paper's analytic test geometries and resolutions
(dx in [0.003, 0.025], Sec. 6-7): the unit circle, the unit sphere, a torus
and a bumpy sphere given by a level set (App. A).  The paper's meshes are not
used; these shapes stand in for them.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

SH_CIRCLE, SH_SPHERE, SH_TORUS, SH_BUMPY = 1, 2, 3, 4
CV_POINT, CV_CIRCLE = 1, 2
BC_DIR1, BC_DIR2, BC_NEU1, BC_NEU2 = 1, 2, 3, 4


@dataclasses.dataclass
class Shape:
    kind: int
    dim: int
    R: float = 1.0            # circle / sphere radius, torus major radius
    rt: float = 0.0           # torus minor radius
    a: Optional[np.ndarray] = None   # bumpy sphere amplitudes a_k
    c: Optional[np.ndarray] = None   # bumpy sphere centres c_k (unit vectors, [K,3])
    amp: float = 0.1
    width: float = 0.05
    seed_point: Sequence[float] = (1.0, 0.0, 0.0)   # a point on S (starts the band search)

    @property
    def K(self) -> int:
        return 0 if self.a is None else int(len(self.a))


@dataclasses.dataclass
class Curve:
    """An interior boundary C: a point, or a circle (centre p, unit normal nu,
    radius rad).  `nu` also orients the two sides: for a circle the side of a
    surface point y is sign((y - cp_C) . nu); for a point in 2D `nu` is the
    unit tangent of S at the point.  `ref` is the circle's angle-0 direction."""
    kind: int
    bc: int
    p: Sequence[float]
    nu: Sequence[float] = (0.0, 0.0, 1.0)
    rad: float = 0.0
    ref: Sequence[float] = (1.0, 0.0, 0.0)
    two_sided: bool = False
    bc_minus: int = 0        # BC type on the minus side (0: the same as bc, the plus side's)
    projected: bool = False  # the projected crossing test (Sec. 4.7) instead of the plain one


@dataclasses.dataclass
class Workload:
    name: str
    shape: Shape
    h: float
    curves: List[Curve]
    m: float
    n: float
    note: str = ""


def circle2d() -> Shape:
    return Shape(SH_CIRCLE, 2, R=1.0, seed_point=(1.0, 0.0, 0.0))


def sphere(R: float = 1.0) -> Shape:
    return Shape(SH_SPHERE, 3, R=R, seed_point=(R, 0.0, 0.0))


def torus(R: float = 1.0, rt: float = 0.4) -> Shape:
    return Shape(SH_TORUS, 3, R=R, rt=rt, seed_point=(R + rt, 0.0, 0.0))


def bumpy_sphere(K: int = 16, seed: int = 0, amp: float = 0.1, width: float = 0.05) -> Shape:
    """rho(w) = 1 + amp * sum_k a_k exp(-|w - c_k|^2 / width), w = x/|x|,
    a_k ~ U[-1, 1], c_k uniform on S^2 (normalised Gaussian triples)."""
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, 1.0, size=K)
    c = rng.normal(size=(K, 3))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    sh = Shape(SH_BUMPY, 3, R=1.0, a=a, c=c, amp=amp, width=width)
    # a surface point in direction +x: rho(e_x) e_x
    ex = np.array([1.0, 0.0, 0.0])
    rho = 1.0 + amp * float(np.sum(a * np.exp(-np.sum((ex - c) ** 2, axis=1) / width)))
    sh.seed_point = (rho, 0.0, 0.0)
    return sh


def bumpy_radius(sh: Shape, w: np.ndarray) -> np.ndarray:
    """rho at unit directions w [...,3] (describes the geometry; used to place
    curves on the surface)."""
    d2 = np.sum((w[..., None, :] - sh.c) ** 2, axis=-1)
    return 1.0 + sh.amp * np.sum(sh.a * np.exp(-d2 / sh.width), axis=-1)


def point_curve(p, bc=BC_DIR1, tangent=(0.0, 0.0, 0.0), two_sided=False) -> Curve:
    return Curve(CV_POINT, bc, tuple(float(v) for v in p), nu=tuple(tangent), two_sided=two_sided)


def circle_on_unit_circle(theta: float, bc=BC_DIR1, two_sided=False) -> Curve:
    """A point C on the unit circle at angle theta; nu = counter-clockwise tangent."""
    return point_curve((math.cos(theta), math.sin(theta), 0.0), bc,
                       tangent=(-math.sin(theta), math.cos(theta), 0.0), two_sided=two_sided)


def latitude_circle(theta: float, bc=BC_DIR1, R: float = 1.0) -> Curve:
    """The circle at polar angle theta on a sphere of radius R (normal +z)."""
    return Curve(CV_CIRCLE, bc, (0.0, 0.0, R * math.cos(theta)), nu=(0.0, 0.0, 1.0),
                 rad=R * math.sin(theta), ref=(1.0, 0.0, 0.0))


def torus_meridian(phi: float, R: float, rt: float, bc=BC_DIR1) -> Curve:
    """The meridian circle of the torus at toroidal angle phi."""
    c, s = math.cos(phi), math.sin(phi)
    return Curve(CV_CIRCLE, bc, (R * c, R * s, 0.0), nu=(-s, c, 0.0), rad=rt, ref=(c, s, 0.0))


def tube_radius(dim: int, h: float, p: int = 3, q: int = 1) -> float:
    """Eq. (3) of the paper (band radius); provided for sizing only."""
    half = (p + 1) / 2.0
    return h * math.sqrt((dim - 1) * half * half + (q + half) ** 2)


def meridian_angles(k: int, seed: int, min_gap: float) -> np.ndarray:
    """k toroidal angles drawn U[0, 2pi) with rejection to a minimum circular gap."""
    rng = np.random.default_rng(seed)
    out: list = []
    tries = 0
    while len(out) < k:
        tries += 1
        if tries > 100000:
            raise RuntimeError("cannot place meridians with that gap")
        a = float(rng.uniform(0.0, 2.0 * math.pi))
        if all(min(abs(a - b), 2 * math.pi - abs(a - b)) >= min_gap for b in out):
            out.append(a)
    return np.sort(np.array(out))


def real_ylm(l: int, m: int, xyz: np.ndarray) -> np.ndarray:
    """Real orthonormal spherical harmonic Y_l^m at the directions of xyz [...,3]
    (input data only: targets and sources are drawn from these)."""
    from scipy.special import sph_harm_y
    r = np.linalg.norm(xyz, axis=-1)
    th = np.arccos(np.clip(xyz[..., 2] / r, -1.0, 1.0))
    ph = np.arctan2(xyz[..., 1], xyz[..., 0])
    if m == 0:
        return np.real(sph_harm_y(l, 0, th, ph))
    y = sph_harm_y(l, abs(m), th, ph)
    if m > 0:
        return math.sqrt(2.0) * (-1) ** m * np.real(y)
    return math.sqrt(2.0) * (-1) ** m * np.imag(y)


# ---------------------------------------------------------------------------
# The five workloads (full sizes) and their small parity-test versions.

def config1(h: float = 0.01, bc: int = BC_DIR1) -> Workload:
    """Unit circle, Dirichlet points u(0)=0, u(pi/2)=1 (Laplace-Beltrami)."""
    return Workload("circle2d", circle2d(), h,
                    [circle_on_unit_circle(0.0, bc), circle_on_unit_circle(math.pi / 2, bc)],
                    m=0.0, n=1.0, note="values 0 at theta=0, 1 at theta=pi/2")


def config2(h: float = 1.0 / 128, bc: int = BC_DIR1) -> Workload:
    """Unit sphere, Dirichlet circles theta=pi/4 (u=0) and 3pi/4 (u=1)."""
    return Workload("sphere_latitudes", sphere(), h,
                    [latitude_circle(math.pi / 4, bc), latitude_circle(3 * math.pi / 4, bc)],
                    m=0.0, n=1.0)


def config3(h: float = 1.0 / 256, ncurves: int = 8, nrhs: int = 64, seed: int = 0,
            min_gap: float = 0.2, bc: int = BC_DIR1):
    """Torus R=1, r=0.4; ncurves meridians at seeded angles; values U[0,1]
    per (curve, rhs)."""
    R, rt = 1.0, 0.4
    ang = meridian_angles(ncurves, seed, min_gap)
    curves = [torus_meridian(float(a), R, rt, bc) for a in ang]
    rng = np.random.default_rng(seed + 1)
    g = rng.uniform(0.0, 1.0, size=(ncurves, nrhs))
    return Workload("torus_batch", torus(R, rt), h, curves, m=0.0, n=1.0), ang, g


def config4(h: float = 1.0 / 256, nsamples: int = 2048, seed: int = 0, bc: int = BC_DIR1):
    """Unit sphere, circle theta=pi/3 with nsamples N(0,1) Dirichlet samples;
    target = sum_{l<=6,m} c_lm Y_lm with c ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    samples = rng.normal(size=nsamples)
    coef = rng.normal(size=49)
    return (Workload("sphere_adjoint", sphere(), h, [latitude_circle(math.pi / 3, bc)], m=0.0, n=1.0),
            samples, coef)


def target_field(coef: np.ndarray, xyz: np.ndarray) -> np.ndarray:
    out = np.zeros(xyz.shape[:-1])
    k = 0
    for l in range(7):
        for m in range(-l, l + 1):
            out += coef[k] * real_ylm(l, m, xyz)
            k += 1
    return out


def config5(h: float = 1.0 / 640, seed: int = 0, bc: int = BC_DIR1) -> Workload:
    """Bumpy sphere, point source at the surface point in direction +z;
    backward-Euler heat step with dt = h, then a Poisson solve."""
    sh = bumpy_sphere(16, seed)
    rz = float(bumpy_radius(sh, np.array([0.0, 0.0, 1.0])))
    return Workload("bumpy_heat", sh, h, [point_curve((0.0, 0.0, rz), bc)], m=1.0, n=-h)


def random_vector(n: int, seed: int, nrhs: int = 1) -> np.ndarray:
    rng = np.random.default_rng(seed)
    if nrhs == 1:
        return rng.uniform(-1.0, 1.0, size=n)
    return rng.uniform(-1.0, 1.0, size=(n, nrhs))
