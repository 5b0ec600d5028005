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
// A point in pixel row j0 of column i crosses the faces c_j (j >= j0) of its column, c_j = 1 where
// rows j and j + 1 differ (c_ny = 1 where the top row is set).  Every point of a pixel sees the same
// count, so it is formed once per pixel: a block takes 8 image columns, splits the rows into 32
// segments, and forms the parity of sum_{j >= j0} c_j for every pixel by a suffix XOR (within each
// segment while walking down it, then across the segments), held as bytes in shared memory; the
// block then writes the grid points of its share of the grid rows whose pixel lies in its columns.
// Images too tall for shared memory, or grids much finer than the image, use one thread per grid
// point walking its ray instead (the same count).
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

constexpr int MP_COLS = 8, MP_SEGS = 32;        // block: image columns x row segments
constexpr int MP_MAX_SMEM = 160 * 1024;          // parity bytes per block: MP_COLS x (ny + 1)
constexpr int MP_MAXK = 2048, MP_MAXL = 1024;    // grid columns / rows one block writes (scan form)

__device__ __forceinline__ int pixel_of(int k, int g, double L, int n) {  // pixel index of grid index k
  const double x = (k + 0.5) * (L / g), h = L / n;
  int i = (int)floor(x / h + 0.5);
  return i < 0 ? 0 : (i > n ? n : i);
}

__global__ void __launch_bounds__(MP_COLS * MP_SEGS) k_ray_parity_scan(
    const double* __restrict__ pp, const double* __restrict__ pn, int nx, int ny, double Lx, double Ly,
    int use_thr, double thr, int gx, int gy, uint8_t* __restrict__ polymer, double* __restrict__ mu_e,
    double* __restrict__ mu_h) {
  extern __shared__ uint8_t par[];  // [MP_COLS][ny + 1]
  __shared__ uint8_t seg_par[MP_SEGS][MP_COLS];
  const int c = threadIdx.x % MP_COLS, sgi = threadIdx.x / MP_COLS;
  const int i0 = blockIdx.x * MP_COLS, i = i0 + c;
  const int rows = ny + 1, W = nx + 1;
  const int seg = (rows + MP_SEGS - 1) / MP_SEGS;
  const int ja = sgi * seg, jb = min(rows, ja + seg);
  uint8_t* col = par + c * rows;
  // 1. within the segment, walking down: loc(j) = c_j ^ loc(j + 1), c_j = img_j ^ img_{j+1}
  uint8_t acc = 0;
  if (i <= nx && ja < jb) {
    bool up = jb < rows ? set_at(pp, pn, use_thr, thr, (int64_t)jb * W + i) : false;  // above the box: unset
    for (int j = jb - 1; j >= ja; --j) {
      const bool here = set_at(pp, pn, use_thr, thr, (int64_t)j * W + i);
      acc ^= (uint8_t)(here != up);
      col[j] = acc;
      up = here;
    }
  }
  seg_par[sgi][c] = acc;
  __syncthreads();
  // 2. across the segments: every row of segment s also crosses the faces of the segments above
  uint8_t carry = 0;
  for (int t = sgi + 1; t < MP_SEGS; ++t) carry ^= seg_par[t][c];
  if (i <= nx && carry)
    for (int j = ja; j < jb; ++j) col[j] ^= 1;
  __syncthreads();
  // 3. the grid points whose pixel column is in [i0, i0 + MP_COLS): grid columns [k0, k1), rows of
  // this block's share (blockIdx.y); pixel indices of its columns and rows formed once into
  // shared memory (the same floor formula as the classification, so the bounds are exact)
  // (one thread finds the column range: FP64 divisions are costly on this part's FP64 pipe)
  __shared__ int krange[2];
  if (threadIdx.x == 0) {
    const int ilast = min(nx, i0 + MP_COLS - 1);
    int a = (int)floor(((i0 - 0.5) * (Lx / nx)) / (Lx / gx) - 0.5);
    int b = (int)ceil(((ilast + 0.5) * (Lx / nx)) / (Lx / gx) + 0.5);
    a = max(0, a - 1);
    b = min(gx, b + 1);
    while (a < b && pixel_of(a, gx, Lx, nx) < i0) ++a;
    while (b > a && pixel_of(b - 1, gx, Lx, nx) > ilast) --b;
    krange[0] = a;
    krange[1] = b;
  }
  __syncthreads();
  const int k0 = krange[0];
  const int nk = min(krange[1] - k0, MP_MAXK);
  const int rows_per = (gy + gridDim.y - 1) / gridDim.y;
  const int l0 = blockIdx.y * rows_per, l1 = min(gy, l0 + rows_per);
  const int nl = min(l1 - l0, MP_MAXL);
  __shared__ int ipix[MP_MAXK], jpix[MP_MAXL];
  for (int t = threadIdx.x; t < nk; t += blockDim.x) ipix[t] = pixel_of(k0 + t, gx, Lx, nx) - i0;
  for (int t = threadIdx.x; t < nl; t += blockDim.x) jpix[t] = pixel_of(l0 + t, gy, Ly, ny);
  __syncthreads();
  if (nk <= 0 || nl <= 0) return;
  for (int t = threadIdx.x; t < nk * nl; t += blockDim.x) {  // nk * nl <= MP_MAXK * MP_MAXL
    const int l = t / nk, kk = t - l * nk;
    const bool inside = par[ipix[kk] * rows + jpix[l]] & 1;
    const int64_t o = (int64_t)(l0 + l) * gx + k0 + kk;
    if (polymer) polymer[o] = inside;
    if (mu_e) mu_e[o] = inside ? MU_LOW : MU_HIGH;
    if (mu_h) mu_h[o] = inside ? MU_HIGH : MU_LOW;
  }
}

ch_status morphology_project(const double* pp, const double* pn, int nx, int ny, double Lx, double Ly,
                             int use_thr, double thr, int gx, int gy, uint8_t* polymer, double* mu_e,
                             double* mu_h, cudaStream_t st) {
  const int64_t G = (int64_t)gx * gy;
  const size_t smem = (size_t)MP_COLS * (ny + 1);
  ProfScope ps(st, K_MORPH, 0, (double)G * (1.0 + 16.0) + 16.0 * (double)(nx + 1) * (ny + 1), 0.0);
  // grid columns per block of 8 image columns: 8 gx / nx (+2 at the edges); rows split over blockIdx.y
  const double kper = (double)MP_COLS * gx / nx + 4.0;
  const int ychunks = (gy + MP_MAXL - 1) / MP_MAXL;
  const int cols_blocks = (nx + 1 + MP_COLS - 1) / MP_COLS;
  const int yblocks = std::max(ychunks, std::min((gy + 63) / 64, (2 * 152 + cols_blocks - 1) / cols_blocks));
  if (smem <= (size_t)MP_MAX_SMEM && kper <= MP_MAXK) {
    CH_CUDA(cudaFuncSetAttribute(k_ray_parity_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, MP_MAX_SMEM));
    k_ray_parity_scan<<<dim3(cols_blocks, yblocks), MP_COLS * MP_SEGS, smem, st>>>(
        pp, pn, nx, ny, Lx, Ly, use_thr, thr, gx, gy, polymer, mu_e, mu_h);
  } else {
    k_ray_parity<<<(unsigned)((G + TPB - 1) / TPB), TPB, 0, st>>>(pp, pn, nx, ny, Lx, Ly, use_thr, thr, gx, gy,
                                                                   polymer, mu_e, mu_h);
  }
  CH_LAUNCHED();
  return CH_OK;
}

}  // namespace ch
