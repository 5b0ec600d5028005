// Morphology -> finite-difference grid projection (Section 5).
//
// Section 5 feeds a simulated morphology to a drift-diffusion device model: the concentration
// field is thresholded into a binary image, the image is treated as an object, and every point of
// a finite-difference grid is classified as inside or outside the object by the parity of the
// number of object faces that a ray from the point crosses; the class sets the carrier
// mobilities at that point.  Here the object is the union of the set pixels, pixel (i, j) being
// the half-open cell of node (i, j) clipped to the box, and the ray runs upward from the point
// (x fixed).  It can only cross horizontal faces: the boundaries between vertically adjacent
// pixels of different value, and the top edge of the box above a set top-row pixel.
//
// One thread per grid point walks its ray through the image column that contains it, counting
// those faces; a warp's points lie in consecutive columns, so every step of the walk is one
// coalesced row segment read.  No scratch memory.
#include <cmath>

#include "ch_internal.cuh"

namespace ch {

constexpr double MU_HIGH = 0.1, MU_LOW = 1e-10;  // m^2 / (V s): Section 5's two mobility values

// pixel (i, j) of the binary image: polymer where phi_p > phi_nfa, or phi_p > threshold
__device__ __forceinline__ bool set_at(const double* pp, const double* pn, int use_thr, double thr, int64_t v) {
  const double a = pp[v];
  return use_thr ? (a > thr) : (a > pn[v]);
}

__global__ void k_ray_parity(const double* __restrict__ pp, const double* __restrict__ pn, int nx, int ny,
                             double Lx, double Ly, int use_thr, double thr, int gx, int gy,
                             uint8_t* __restrict__ polymer, double* __restrict__ mu_e, double* __restrict__ mu_h) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)gx * gy) return;
  const int k = (int)(t % gx), l = (int)(t / gx);
  // grid point: centre of cell (k, l) of a uniform gx x gy grid of the box
  const double x = (k + 0.5) * (Lx / gx), y = (l + 0.5) * (Ly / gy);
  const double hx = Lx / nx, hy = Ly / ny;
  // the pixel column and row containing the point (pixel i spans [(i - 1/2) hx, (i + 1/2) hx))
  int i = (int)floor(x / hx + 0.5), j0 = (int)floor(y / hy + 0.5);
  i = i < 0 ? 0 : (i > nx ? nx : i);
  j0 = j0 < 0 ? 0 : (j0 > ny ? ny : j0);
  const int64_t W = nx + 1;
  // faces above the point: between rows j and j + 1 for j >= j0, then the box's top edge
  bool below = set_at(pp, pn, use_thr, thr, (int64_t)j0 * W + i);
  int crossings = 0;
  for (int j = j0; j < ny; ++j) {
    const bool up = set_at(pp, pn, use_thr, thr, (int64_t)(j + 1) * W + i);
    crossings += below != up;
    below = up;
  }
  crossings += below;
  const bool inside = crossings & 1;
  if (polymer) polymer[t] = inside;
  if (mu_e) mu_e[t] = inside ? MU_LOW : MU_HIGH;   // polymer phase: electrons slow, holes fast
  if (mu_h) mu_h[t] = inside ? MU_HIGH : MU_LOW;
}

ch_status morphology_project(const double* pp, const double* pn, int nx, int ny, double Lx, double Ly,
                             int use_thr, double thr, int gx, int gy, uint8_t* polymer, double* mu_e,
                             double* mu_h, cudaStream_t st) {
  const int64_t G = (int64_t)gx * gy;
  ProfScope ps(st, K_MORPH, 0, (double)G * (1.0 + 16.0) + 16.0 * (double)(nx + 1) * (ny + 1), 0.0);
  k_ray_parity<<<(unsigned)((G + TPB - 1) / TPB), TPB, 0, st>>>(pp, pn, nx, ny, Lx, Ly, use_thr, thr, gx, gy,
                                                                 polymer, mu_e, mu_h);
  CH_LAUNCHED();
  return CH_OK;
}

}  // namespace ch
