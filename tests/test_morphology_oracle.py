"""Pins of the morphology-to-grid projection oracle (Section 5), CPU only.

The oracle classifies a grid point by the image pixel that contains it.  Section 5 classifies it
by the parity of the object faces that a ray from the point to the top of the domain crosses;
the first test builds the object's boundary faces from the image and counts those crossings in
plain loops, so the definition is checked against the paper's method.
"""
import numpy as np
import pytest

from oracle import morphology_oracle as mo


def boundary_faces(img, Lx, Ly):
    """Horizontal faces of the union of set pixels (pixel (i, j) centred on node (i, j), clipped to
    the box): between vertically adjacent pixels of different value, and the box's top edge above a
    set pixel of the top row.  Faces parallel to an upward ray (vertical ones) are never crossed."""
    ny1, nx1 = img.shape
    hx, hy = Lx / (nx1 - 1), Ly / (ny1 - 1)
    faces = []  # (y, x0, x1)
    for i in range(nx1):
        x0, x1 = max((i - 0.5) * hx, 0.0), min((i + 0.5) * hx, Lx)
        for j in range(ny1 - 1):
            if img[j, i] != img[j + 1, i]:
                faces.append(((j + 0.5) * hy, x0, x1))
        if img[ny1 - 1, i]:
            faces.append((Ly, x0, x1))
    return faces


def ray_parity(faces, x, y):
    """Number of faces above (x, y) met by the upward ray x = const, modulo 2 (half-open in x)."""
    n = 0
    for fy, x0, x1 in faces:
        if fy > y and x0 <= x < x1:
            n += 1
    return n % 2 == 1


@pytest.mark.parametrize("seed,nx,ny,gx,gy", [(0, 12, 7, 31, 17), (1, 20, 10, 53, 29), (2, 5, 9, 13, 23)])
def test_classification_equals_ray_crossing_parity(seed, nx, ny, gx, gy):
    rng = np.random.default_rng(seed)
    Lx, Ly = 10.0, 2.5
    N = (nx + 1) * (ny + 1)
    pp, pn = rng.random(N), rng.random(N)
    img = mo.binary_image(pp, pn, nx, ny)
    X, Y = mo.grid_points(gx, gy, Lx, Ly)
    got = mo.classify(img, X, Y, Lx, Ly)
    faces = boundary_faces(img, Lx, Ly)
    ref = np.array([[ray_parity(faces, X[l, k], Y[l, k]) for k in range(gx)] for l in range(gy)])
    np.testing.assert_array_equal(got, ref)
    assert 0 < got.sum() < got.size  # both phases present


def test_disk_morphology():
    """A polymer disk of radius 0.8 centred in [0, 4] x [0, 2]: grid points farther than one pixel
    diagonal from the circle are classified by the circle itself."""
    nx, ny, Lx, Ly = 80, 40, 4.0, 2.0
    x = np.tile(np.arange(nx + 1) * (Lx / nx), ny + 1)
    y = np.repeat(np.arange(ny + 1) * (Ly / ny), nx + 1)
    r = np.hypot(x - 2.0, y - 1.0)
    pp = np.where(r < 0.8, 0.9, 0.1)
    polymer, mu_e, mu_h = mo.project(pp, 1.0 - pp, nx, ny, Lx, Ly, 97, 51)
    X, Y = mo.grid_points(97, 51, Lx, Ly)
    rr = np.hypot(X - 2.0, Y - 1.0)
    diag = np.hypot(Lx / nx, Ly / ny)
    assert polymer[rr < 0.8 - diag].all() and not polymer[rr > 0.8 + diag].any()
    np.testing.assert_array_equal(mu_e[polymer], mo.MU_LOW)
    np.testing.assert_array_equal(mu_h[polymer], mo.MU_HIGH)
    np.testing.assert_array_equal(mu_e[~polymer], mo.MU_HIGH)
    np.testing.assert_array_equal(mu_h[~polymer], mo.MU_LOW)


def test_threshold_readings():
    """phi_p > phi_nfa by default; an explicit threshold compares phi_p alone."""
    pp = np.array([0.6, 0.3, 0.45, 0.2])
    pn = np.array([0.2, 0.5, 0.5, 0.1])
    np.testing.assert_array_equal(mo.binary_image(pp, pn, 1, 1).ravel(), [True, False, False, True])
    np.testing.assert_array_equal(mo.binary_image(pp, pn, 1, 1, threshold=0.4).ravel(), [True, False, True, False])


def test_grid_aligned_with_pixels_takes_the_pixel_of_each_node():
    """When the grid points are the nodes' own positions shifted by less than half a pixel, each
    point takes its node's value: the image itself comes back."""
    rng = np.random.default_rng(3)
    nx, ny, Lx, Ly = 9, 6, 9.0, 6.0
    img = rng.random((ny + 1, nx + 1)) > 0.5
    X, Y = np.meshgrid(np.arange(nx + 1) + 0.2, np.arange(ny + 1) - 0.3 * (np.arange(ny + 1) > 0), indexing="xy")
    np.testing.assert_array_equal(mo.classify(img, X, Y, Lx, Ly), img)


def test_grid_points_are_cell_centres():
    X, Y = mo.grid_points(4, 2, 10.0, 2.5)
    np.testing.assert_allclose(X[0], [1.25, 3.75, 6.25, 8.75], rtol=1e-15)
    np.testing.assert_allclose(Y[:, 0], [0.625, 1.875], rtol=1e-15)
