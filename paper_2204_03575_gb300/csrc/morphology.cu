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
// For a point in pixel row j0 of column i the crossings are c_j = img_j xor img_{j+1} for
// j0 <= j < ny and c_ny = img_ny, and their parity telescopes:
//   c_j0 xor ... xor c_ny = (img_j0 xor img_{j0+1}) xor ... xor (img_{ny-1} xor img_ny) xor img_ny
//                         = img_j0,
// the value of the pixel that holds the point.  So the kernel classifies each point by reading
// that one pixel -- a gather whose cost is the writes of the three output maps -- instead of
// summing the faces along the ray.  (The test suite checks the classes bit for bit against a CPU
// oracle that is itself pinned to an explicit crossing count.)
#include <algorithm>
#include <cmath>

#include "ch_internal.cuh"

namespace ch {

constexpr double MU_HIGH = 0.1, MU_LOW = 1e-10;  // m^2 / (V s): Section 5's two mobility values

// pixel (i, j) of the binary image: polymer where phi_p > phi_nfa, or phi_p > threshold
__device__ __forceinline__ bool set_at(const double* pp, const double* pn, int use_thr, double thr, int64_t v) {
  const double a = pp[v];
  return use_thr ? (a > thr) : (a > pn[v]);
}

// Pixel index of grid index k along one axis (g grid cells and n image cells over a box of length
// L): the point (k + 1/2) L / g lies in pixel floor(x / (L / n) + 1/2), clamped to [0, n] -- the
// classification is defined by this FP64 evaluation.  In exact arithmetic the rounded value is
// t / (2g) with t = (2k + 1) n + g.  Unless 2g divides t, that value lies at least 1 / (2g) from
// an integer, while the FP64 evaluation (four correctly rounded operations) stays within
// n x 2^-50 of it; for n g <= 1e12 the floor is then the integer quotient, which `exact` takes.
// Exact ties (and larger sizes) use the FP64 formula itself.
__device__ __forceinline__ int pixel_index(int k, int g, double L, int n, bool exact) {
  if (exact) {
    const long long t = (2LL * k + 1) * n + g, g2 = 2LL * g;
    const long long q = t / g2;
    if (q * g2 != t) return (int)(q > n ? n : q);  // t > 0, so q >= 0
  }
  const double x = (k + 0.5) * (L / g), h = L / n;
  const int i = (int)floor(x / h + 0.5);
  return i < 0 ? 0 : (i > n ? n : i);
}

constexpr int MP_TX = 256, MP_TY = 8;  // grid points per block: MP_TX columns x MP_TY rows

// One block per MP_TX x MP_TY patch of the grid: the pixel column of every grid column and the
// pixel row of every grid row are formed once per block, then each thread classifies its column's
// MP_TY points (the row loads in flight together, stores coalesced along each grid row).
__global__ void __launch_bounds__(MP_TX) k_classify(const double* __restrict__ pp, const double* __restrict__ pn,
                                                    int nx, int ny, double Lx, double Ly, int use_thr, double thr,
                                                    int gx, int gy, int exact, uint8_t* __restrict__ polymer,
                                                    double* __restrict__ mu_e, double* __restrict__ mu_h) {
  __shared__ long long rowbase[MP_TY];  // first pixel of each grid row's pixel row
  const int nbx = (gx + MP_TX - 1) / MP_TX;  // blocks along a grid row (one grid dimension: any gy)
  const int bx = (int)(blockIdx.x % (unsigned)nbx), by = (int)(blockIdx.x / (unsigned)nbx);
  const int k = bx * MP_TX + threadIdx.x, l0 = by * MP_TY;
  if (threadIdx.x < MP_TY && l0 + (int)threadIdx.x < gy)
    rowbase[threadIdx.x] = (long long)pixel_index(l0 + threadIdx.x, gy, Ly, ny, exact) * (nx + 1);
  const int i = k < gx ? pixel_index(k, gx, Lx, nx, exact) : 0;
  __syncthreads();
  if (k >= gx) return;
  const int rows = min(MP_TY, gy - l0);
  bool inside[MP_TY];
#pragma unroll
  for (int r = 0; r < MP_TY; ++r) inside[r] = r < rows && set_at(pp, pn, use_thr, thr, rowbase[r] + i);
#pragma unroll
  for (int r = 0; r < MP_TY; ++r) {
    if (r >= rows) break;
    const int64_t o = (int64_t)(l0 + r) * gx + k;
    if (polymer) polymer[o] = inside[r];
    if (mu_e) mu_e[o] = inside[r] ? MU_LOW : MU_HIGH;  // polymer phase: electrons slow, holes fast
    if (mu_h) mu_h[o] = inside[r] ? MU_HIGH : MU_LOW;
  }
}

ch_status morphology_project(const double* pp, const double* pn, int nx, int ny, double Lx, double Ly,
                             int use_thr, double thr, int gx, int gy, uint8_t* polymer, double* mu_e,
                             double* mu_h, cudaStream_t st) {
  const int64_t G = (int64_t)gx * gy;
  // algorithmic bytes: the three maps written once, the image's fields read once
  ProfScope ps(st, K_MORPH, 0, (double)G * (1.0 + 16.0) + (use_thr ? 8.0 : 16.0) * (double)(nx + 1) * (ny + 1),
               0.0);
  const int exact = (double)nx * gx <= 1e12 && (double)ny * gy <= 1e12;
  const int64_t nblocks = (int64_t)((gx + MP_TX - 1) / MP_TX) * ((gy + MP_TY - 1) / MP_TY);  // < 2^31: G < 2e9
  k_classify<<<(unsigned)nblocks, MP_TX, 0, st>>>(pp, pn, nx, ny, Lx, Ly, use_thr, thr, gx, gy, exact, polymer,
                                                  mu_e, mu_h);
  CH_LAUNCHED();
  return CH_OK;
}

}  // namespace ch
