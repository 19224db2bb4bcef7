"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds problem *definitions* only: the embedded shapes, the
manufactured solution and its derivatives, and the Gaussian-bump right-hand
sides.  It contains none of the cut-cell method's arithmetic (no quadrature,
merging, stencils, fitting or solver steps), so both sides can draw the same
inputs from it without sharing any of the method.

Conventions
-----------
* The box is [0,1]^3, cells per axis ``n``, h = 1/n.
* A shape is an axis-aligned ellipsoid ``(centre[3], semi_axes[3])``; a sphere
  has three equal semi-axes.  The fluid domain is the box minus the union of
  the shapes.
* Boundary kinds: 0 = Dirichlet, 1 = Neumann.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

DIRICHLET = 0
NEUMANN = 1


@dataclass
class Problem:
    """A cut-cell Poisson problem: geometry plus boundary kinds."""

    n: int
    shapes: list  # list of (centre ndarray(3), semi ndarray(3))
    shape_bc: int = DIRICHLET
    box_bc: tuple = (DIRICHLET,) * 6  # faces x-,x+,y-,y+,z-,z+
    name: str = ""
    bumps: dict | None = field(default=None)

    def with_n(self, n: int) -> "Problem":
        return Problem(n, self.shapes, self.shape_bc, self.box_bc, self.name, self.bumps)


# ---------------------------------------------------------------- geometry
def sphere_problem(n: int, radius: float = 0.25) -> Problem:
    """Box minus a sphere of the given radius centred at (1/2,1/2,1/2), Dirichlet everywhere."""
    c = np.array([0.5, 0.5, 0.5])
    a = np.array([radius] * 3)
    return Problem(n, [(c, a)], DIRICHLET, (DIRICHLET,) * 6, f"sphere_r{radius}")


def ellipsoids_problem(n: int, seed: int, count: int = 3) -> Problem:
    """Box minus ``count`` axis-aligned ellipsoids drawn from ``default_rng(seed)``.

    Draw order per ellipsoid: centre ~ U[0.3,0.7]^3, then semi-axes ~ U[0.1,0.25]^3.
    Neumann on the ellipsoids, Dirichlet on the box.
    """
    rng = np.random.default_rng(seed)
    shapes = []
    for _ in range(count):
        c = rng.uniform(0.3, 0.7, 3)
        a = rng.uniform(0.1, 0.25, 3)
        shapes.append((c, a))
    return Problem(n, shapes, NEUMANN, (DIRICHLET,) * 6, f"ellipsoids{count}_seed{seed}")


def batch_problem(seed: int, sizes=(64, 96, 128, 160, 192)) -> Problem:
    """One solve of the batched workload: size from ``sizes``, 1-4 spheres/ellipsoids.

    Radii ~ U[0.08,0.25], centres ~ U[0.3,0.7]^3; spheres and ellipsoids equally
    likely; Neumann on the shapes; Gaussian-bump RHS parameters attached.
    """
    rng = np.random.default_rng(10_000 + seed)
    n = int(rng.choice(np.array(sizes)))
    k = int(rng.integers(1, 5))
    shapes = []
    for _ in range(k):
        c = rng.uniform(0.3, 0.7, 3)
        if rng.uniform() < 0.5:
            a = np.full(3, rng.uniform(0.08, 0.25))
        else:
            a = rng.uniform(0.08, 0.25, 3)
        shapes.append((c, a))
    p = Problem(n, shapes, NEUMANN, (DIRICHLET,) * 6, f"batch_seed{seed}")
    p.bumps = gaussian_bumps(shapes, seed=20_000 + seed)
    return p


def guess_problem(n: int, seed: int, bump_seed: int | None = None) -> Problem:
    """One pair of the learned-guess workload: the three-ellipsoid geometry
    drawn like ``ellipsoids_problem`` but with 2-4 ellipsoids (semi-axes
    U[0.1,0.25], centres U[0.3,0.7]^3), Neumann on the ellipsoids, Dirichlet on
    the box, and the manufactured right-hand side plus 20 Gaussian bumps (drawn
    from ``bump_seed`` when given, so that one geometry can carry several)."""
    rng = np.random.default_rng(30_000 + seed)
    k = int(rng.integers(2, 5))
    shapes = []
    for _ in range(k):
        c = rng.uniform(0.3, 0.7, 3)
        a = rng.uniform(0.1, 0.25, 3)
        shapes.append((c, a))
    p = Problem(n, shapes, NEUMANN, (DIRICHLET,) * 6, f"guess_seed{seed}")
    p.bumps = gaussian_bumps(shapes, seed=40_000 + (seed if bump_seed is None else 1_000_000 + bump_seed))
    return p


def inside_any(shapes, x, y, z):
    """True where the point lies inside (or on) any shape."""
    m = np.zeros(np.broadcast(x, y, z).shape, dtype=bool)
    for c, a in shapes:
        m |= ((x - c[0]) / a[0]) ** 2 + ((y - c[1]) / a[1]) ** 2 + ((z - c[2]) / a[2]) ** 2 <= 1.0
    return m


# ------------------------------------------------------- manufactured solution
TWO_PI = 2.0 * math.pi


def phi_exact(x, y, z):
    """phi = sin(2 pi x) sin(2 pi y) sin(2 pi z) + exp(x+y+z)/10."""
    return np.sin(TWO_PI * x) * np.sin(TWO_PI * y) * np.sin(TWO_PI * z) + np.exp(x + y + z) / 10.0


def lap_phi_exact(x, y, z):
    """Laplacian of phi_exact: -12 pi^2 sin sin sin + 0.3 exp(x+y+z)."""
    return (-3.0 * TWO_PI ** 2) * np.sin(TWO_PI * x) * np.sin(TWO_PI * y) * np.sin(TWO_PI * z) + 0.3 * np.exp(x + y + z)


def grad_phi_exact(x, y, z):
    """Gradient of phi_exact as a tuple of three arrays."""
    sx, sy, sz = np.sin(TWO_PI * x), np.sin(TWO_PI * y), np.sin(TWO_PI * z)
    cx, cy, cz = np.cos(TWO_PI * x), np.cos(TWO_PI * y), np.cos(TWO_PI * z)
    e = np.exp(x + y + z) / 10.0
    return (TWO_PI * cx * sy * sz + e, TWO_PI * sx * cy * sz + e, TWO_PI * sx * sy * cz + e)


# --------------------------------------------------------------- bump RHS
def gaussian_bumps(shapes, seed: int, count: int = 20) -> dict:
    """Parameters of sum_k a_k exp(-|x-c_k|^2 / (2 w_k^2)).

    a_k ~ N(0,1), w_k ~ U[0.02,0.1], c_k uniform in the fluid domain (rejection
    sampled against the shapes).
    """
    rng = np.random.default_rng(seed)
    amp = rng.normal(0.0, 1.0, count)
    width = rng.uniform(0.02, 0.1, count)
    centres = np.zeros((count, 3))
    k = 0
    while k < count:
        p = rng.uniform(0.0, 1.0, 3)
        if not inside_any(shapes, p[0], p[1], p[2]):
            centres[k] = p
            k += 1
    return {"amp": amp, "width": width, "centre": centres}


def bump_field(b: dict, x, y, z):
    """Evaluate the Gaussian-bump sum at points."""
    out = np.zeros(np.broadcast(x, y, z).shape)
    for a, w, c in zip(b["amp"], b["width"], b["centre"]):
        r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2
        out = out + a * np.exp(-r2 / (2.0 * w * w))
    return out


def rhs_field(problem: Problem):
    """Right-hand side f(x,y,z): Laplacian of phi_exact plus the bump sum if any."""
    if problem.bumps is None:
        return lap_phi_exact
    b = problem.bumps
    return lambda x, y, z: lap_phi_exact(x, y, z) + bump_field(b, x, y, z)


# ------------------------------------------------------ separable forms
def _sin2pi(x):
    return np.sin(TWO_PI * x)


def phi_terms():
    """phi_exact as a sum of separable products: [(coef, (fx, fy, fz))]."""
    return [(1.0, (_sin2pi, _sin2pi, _sin2pi)), (0.1, (np.exp, np.exp, np.exp))]


def rhs_terms(problem: Problem):
    """f = Lap phi_exact (+ bumps) as a sum of separable products."""
    terms = [(-3.0 * TWO_PI ** 2, (_sin2pi, _sin2pi, _sin2pi)), (0.3, (np.exp, np.exp, np.exp))]
    if problem.bumps is not None:
        b = problem.bumps
        for a, w, c in zip(b["amp"], b["width"], b["centre"]):
            fs = tuple((lambda x, cc=cc, ww=w: np.exp(-(x - cc) ** 2 / (2.0 * ww * ww))) for cc in c)
            terms.append((float(a), fs))
    return terms


def eval_terms(terms, x, y, z):
    out = 0.0
    for coef, (fx, fy, fz) in terms:
        out = out + coef * fx(x) * fy(y) * fz(z)
    return out
