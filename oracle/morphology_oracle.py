"""Plain CPU oracle of the morphology-to-grid projection of Section 5.

TEST INFRASTRUCTURE ONLY: imported by the test suite; the library never uses it and shares no
code with it.

Section 5 turns a simulated morphology into the input of a drift-diffusion device model: the
concentration field is thresholded into a binary image, the image is meshed as an object, and
every point of a finite-difference grid is classified as inside or outside the object by the
parity of the number of object faces a ray from the point crosses; the class sets the carrier
mobilities at that point.  The classification reaches a result with a plain definition -- the
point is inside exactly when the image pixel that contains it is set -- and that definition is
what this module computes.  (tests/test_morphology_oracle.py checks it against a brute-force
crossing count.)

Readings of points the paper leaves open:
  M1 threshold: a node belongs to the polymer phase when phi_p > phi_nfa (the dominant of the
     two solid components); ``threshold`` overrides it with phi_p > threshold;
  M2 the binary image has one pixel per mesh node of an nx x ny 2D mesh: node (i, j) owns the
     half-open cell [(i - 1/2) hx, (i + 1/2) hx) x [(j - 1/2) hy, (j + 1/2) hy), clipped to the box;
  M3 the finite-difference grid has gx x gy points at the centres of a uniform gx x gy cell grid
     of the same box;
  M4 mobilities (Section 5): polymer phase electrons 1e-10, holes 0.1 m^2/(V s); the other phase
     the opposite.
"""
from __future__ import annotations

import numpy as np

MU_HIGH, MU_LOW = 0.1, 1e-10  # m^2 / (V s), Section 5


def binary_image(phi_p: np.ndarray, phi_nfa: np.ndarray, nx: int, ny: int, threshold=None):
    """(ny + 1, nx + 1) bool image of the polymer phase from nodal fields (node i + (nx + 1) j)."""
    pp = np.asarray(phi_p, dtype=np.float64).reshape(ny + 1, nx + 1)
    if threshold is None:
        pn = np.asarray(phi_nfa, dtype=np.float64).reshape(ny + 1, nx + 1)
        return pp > pn
    return pp > threshold


def grid_points(gx: int, gy: int, Lx: float, Ly: float):
    """Centres of a uniform gx x gy cell grid of [0, Lx] x [0, Ly] (reading M3): (gy, gx) arrays."""
    x = (np.arange(gx) + 0.5) * (Lx / gx)
    y = (np.arange(gy) + 0.5) * (Ly / gy)
    return np.meshgrid(x, y, indexing="xy")


def classify(image: np.ndarray, X: np.ndarray, Y: np.ndarray, Lx: float, Ly: float):
    """Polymer (True) / other (False) at the points (X, Y): the value of the pixel that contains
    each point (reading M2: pixel (i, j) is centred on node (i, j), half-open)."""
    ny1, nx1 = image.shape
    hx, hy = Lx / (nx1 - 1), Ly / (ny1 - 1)
    i = np.clip(np.floor(X / hx + 0.5).astype(np.int64), 0, nx1 - 1)
    j = np.clip(np.floor(Y / hy + 0.5).astype(np.int64), 0, ny1 - 1)
    return image[j, i]


def mobilities(polymer: np.ndarray):
    """(electron, hole) mobility maps (reading M4)."""
    mu_e = np.where(polymer, MU_LOW, MU_HIGH)
    mu_h = np.where(polymer, MU_HIGH, MU_LOW)
    return mu_e, mu_h


def project(phi_p, phi_nfa, nx: int, ny: int, Lx: float, Ly: float, gx: int, gy: int, threshold=None):
    """The whole projection: binary image -> classified grid -> mobility maps."""
    img = binary_image(phi_p, phi_nfa, nx, ny, threshold)
    X, Y = grid_points(gx, gy, Lx, Ly)
    polymer = classify(img, X, Y, Lx, Ly)
    mu_e, mu_h = mobilities(polymer)
    return polymer, mu_e, mu_h
