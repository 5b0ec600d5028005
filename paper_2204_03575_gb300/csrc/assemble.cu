// Mesh generation, P1 assembly, explicit loads and the block operator of Eq. (14).
//
// Everything is node-centric ("gather"): the thread of node i visits the simplices or
// boundary facets incident to i in increasing index order and adds their contributions,
// so every sum has a fixed order and results are bitwise reproducible (no atomics).
#include <cmath>

#include "ch_internal.cuh"

namespace ch {

// ---------------------------------------------------------------- mesh (Section 4)
__global__ void k_fill_int(int* a, int n, int v) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

__global__ void k_mesh_nodes(ch_params p, int N, int node_off, double* coords) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const int i = n % (p.nx + 1);
  const int j = (n / (p.nx + 1)) % (p.ny + 1);
  const int g = node_off + n;
  if (p.dim == 2) {
    coords[2 * g + 0] = i * (p.Lx / p.nx);
    coords[2 * g + 1] = j * (p.Ly / p.ny);
  } else {
    const int k = n / ((p.nx + 1) * (p.ny + 1));
    coords[3 * g + 0] = i * (p.Lx / p.nx);
    coords[3 * g + 1] = j * (p.Ly / p.ny);
    coords[3 * g + 2] = k * (p.Lz / p.nz);
  }
}

// 2D: cell c = i + nx j -> triangles 2c = (v00, v10, v11), 2c+1 = (v00, v11, v01).
// 3D: hexahedron c -> the 6 Kuhn tetrahedra v000 -> +e_a -> +e_a+e_b -> v111 over the
// permutations (a,b,c) of the axes, in lexicographic order of the permutation.
__global__ void k_mesh_elems(ch_params p, int E, int node_off, int* el) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  if (p.dim == 2) {
    const int c = e >> 1, i = c % p.nx, j = c / p.nx;
    const int v00 = node_off + i + (p.nx + 1) * j, v10 = v00 + 1, v01 = v00 + p.nx + 1, v11 = v01 + 1;
    if ((e & 1) == 0) {
      el[3 * e] = v00; el[3 * e + 1] = v10; el[3 * e + 2] = v11;
    } else {
      el[3 * e] = v00; el[3 * e + 1] = v11; el[3 * e + 2] = v01;
    }
  } else {
    const int c = e / 6, t = e % 6;
    const int i = c % p.nx, j = (c / p.nx) % p.ny, k = c / (p.nx * p.ny);
    const int s[3] = {1, p.nx + 1, (p.nx + 1) * (p.ny + 1)};
    const int perm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    const int v0 = node_off + i + s[1] * j + s[2] * k;
    el[4 * e + 0] = v0;
    el[4 * e + 1] = v0 + s[perm[t][0]];
    el[4 * e + 2] = v0 + s[perm[t][0]] + s[perm[t][1]];
    el[4 * e + 3] = v0 + s[0] + s[1] + s[2];
  }
}

// Boundary facets of the Kuhn / diagonal split on y = 0 (bottom) and y = Ly (top).
__global__ void k_mesh_facets(ch_params p, int F, int node_off, int* bot, int* top) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= F) return;
  if (p.dim == 2) {
    const int b = node_off + f, t = node_off + p.ny * (p.nx + 1) + f;
    bot[2 * f] = b; bot[2 * f + 1] = b + 1;
    top[2 * f] = t; top[2 * f + 1] = t + 1;
  } else {
    const int q = f >> 1, i = q % p.nx, k = q / p.nx;
    const int sx = 1, sz = (p.nx + 1) * (p.ny + 1);
    const int b = node_off + i + sz * k;                      // (i, 0, k)
    const int t = node_off + i + (p.nx + 1) * p.ny + sz * k;  // (i, ny, k)
    if ((f & 1) == 0) {
      bot[3 * f] = b; bot[3 * f + 1] = b + sx; bot[3 * f + 2] = b + sx + sz;
      top[3 * f] = t; top[3 * f + 1] = t + sx; top[3 * f + 2] = t + sx + sz;
    } else {
      bot[3 * f] = b; bot[3 * f + 1] = b + sz; bot[3 * f + 2] = b + sx + sz;
      top[3 * f] = t; top[3 * f + 1] = t + sz; top[3 * f + 2] = t + sx + sz;
    }
  }
}

// |T| and barycentric gradients: lambda_{1..d} = J^{-1}(x - x_0), J = [x_1-x_0, ..., x_d-x_0].
template <int D>
__device__ __forceinline__ double simplex_geo(const double* coords, const int* v, double g[D + 1][D]);

template <>
__device__ __forceinline__ double simplex_geo<2>(const double* X, const int* v, double g[3][2]) {
  const double x0 = X[2 * v[0]], y0 = X[2 * v[0] + 1];
  const double j00 = X[2 * v[1]] - x0, j10 = X[2 * v[1] + 1] - y0;
  const double j01 = X[2 * v[2]] - x0, j11 = X[2 * v[2] + 1] - y0;
  const double det = j00 * j11 - j01 * j10;
  const double id = 1.0 / det;
  g[1][0] = j11 * id;  g[1][1] = -j01 * id;
  g[2][0] = -j10 * id; g[2][1] = j00 * id;
  g[0][0] = -(g[1][0] + g[2][0]);
  g[0][1] = -(g[1][1] + g[2][1]);
  return 0.5 * fabs(det);
}

template <>
__device__ __forceinline__ double simplex_geo<3>(const double* X, const int* v, double g[4][3]) {
  double e[3][3];
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c) e[a][c] = X[3 * v[a + 1] + c] - X[3 * v[0] + c];
  // rows of J^{-1}: (e2 x e3, e3 x e1, e1 x e2) / det
  double r[3][3];
  for (int a = 0; a < 3; ++a) {
    const double* u = e[(a + 1) % 3];
    const double* w = e[(a + 2) % 3];
    r[a][0] = u[1] * w[2] - u[2] * w[1];
    r[a][1] = u[2] * w[0] - u[0] * w[2];
    r[a][2] = u[0] * w[1] - u[1] * w[0];
  }
  const double det = e[0][0] * r[0][0] + e[0][1] * r[0][1] + e[0][2] * r[0][2];
  const double id = 1.0 / det;
  for (int c = 0; c < 3; ++c) {
    g[1][c] = r[0][c] * id;
    g[2][c] = r[1][c] * id;
    g[3][c] = r[2][c] * id;
    g[0][c] = -(g[1][c] + g[2][c] + g[3][c]);
  }
  return fabs(det) / 6.0;
}

template <int D>
__global__ void k_elem_vol(const double* X, const int* el, int E, double* vol) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= E) return;
  double g[D + 1][D];
  vol[e] = simplex_geo<D>(X, el + (D + 1) * e, g);
}

// facet measure: segment length (2D) or triangle area (3D)
template <int D>
__global__ void k_facet_vol(const double* X, const int* f, int F, double* vol) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= F) return;
  if (D == 2) {
    const double dx = X[2 * f[2 * q + 1]] - X[2 * f[2 * q]];
    const double dy = X[2 * f[2 * q + 1] + 1] - X[2 * f[2 * q] + 1];
    vol[q] = sqrt(dx * dx + dy * dy);
  } else {
    double u[3], w[3];
    for (int c = 0; c < 3; ++c) {
      u[c] = X[3 * f[3 * q + 1] + c] - X[3 * f[3 * q] + c];
      w[c] = X[3 * f[3 * q + 2] + c] - X[3 * f[3 * q] + c];
    }
    const double cx = u[1] * w[2] - u[2] * w[1], cy = u[2] * w[0] - u[0] * w[2],
                 cz = u[0] * w[1] - u[1] * w[0];
    vol[q] = 0.5 * sqrt(cx * cx + cy * cy + cz * cz);
  }
}

// counts of one box mesh
static void box_counts(const ch_params& p, int* N, int* E, int* F) {
  if (p.dim == 2) {
    *N = (p.nx + 1) * (p.ny + 1);
    *E = 2 * p.nx * p.ny;
    *F = p.nx;
  } else {
    *N = (p.nx + 1) * (p.ny + 1) * (p.nz + 1);
    *E = 6 * p.nx * p.ny * p.nz;
    *F = 2 * p.nx * p.nz;
  }
}

// The mesh of every run, laid out one after another: run r owns nodes [run_off[r], run_off[r+1]),
// its elements and boundary facets follow those of run r-1 and reference only its own nodes, so
// the union is a disjoint set of box meshes (one run: the plain mesh).
ch_status mesh_build(ch_mesh_s* m, cudaStream_t st) {
  const int R = (int)m->runs.size();
  const int d = m->runs[0].dim;
  m->dim = d;
  m->p = m->runs[0];
  m->run_off.assign(R + 1, 0);
  std::vector<int> eoff(R + 1, 0), foff(R + 1, 0);
  for (int r = 0; r < R; ++r) {
    int n, e, f;
    box_counts(m->runs[r], &n, &e, &f);
    if ((int64_t)m->run_off[r] + n > 2000000000LL) {
      set_error("batched mesh too large for int32 indexing");
      return CH_ERR_ARG;
    }
    m->run_off[r + 1] = m->run_off[r] + n;
    eoff[r + 1] = eoff[r] + e;
    foff[r + 1] = foff[r] + f;
  }
  m->N = m->run_off[R];
  m->E = eoff[R];
  m->Fb = m->Ft = foff[R];
  CH_TRY(m->mem.get(&m->coords, (size_t)m->N * d));
  CH_TRY(m->mem.get(&m->elems, (size_t)m->E * (d + 1)));
  CH_TRY(m->mem.get(&m->bot, (size_t)m->Fb * d));
  CH_TRY(m->mem.get(&m->top, (size_t)m->Ft * d));
  CH_TRY(m->mem.get(&m->vol, (size_t)m->E));
  CH_TRY(m->mem.get(&m->bvol, (size_t)m->Fb));
  CH_TRY(m->mem.get(&m->tvol, (size_t)m->Ft));
  CH_TRY(m->mem.get(&m->node_run, (size_t)m->N));
  CH_TRY(m->mem.get(&m->run_off_d, (size_t)R + 1));
  for (int r = 0; r < R; ++r) {
    const ch_params& p = m->runs[r];
    const int n = m->run_off[r + 1] - m->run_off[r], e = eoff[r + 1] - eoff[r], f = foff[r + 1] - foff[r];
    k_mesh_nodes<<<blocks_for(n), TPB, 0, st>>>(p, n, m->run_off[r], m->coords);
    k_mesh_elems<<<blocks_for(e), TPB, 0, st>>>(p, e, m->run_off[r], m->elems + (size_t)eoff[r] * (d + 1));
    k_mesh_facets<<<blocks_for(f), TPB, 0, st>>>(p, f, m->run_off[r], m->bot + (size_t)foff[r] * d,
                                                  m->top + (size_t)foff[r] * d);
    k_fill_int<<<blocks_for(n), TPB, 0, st>>>(m->node_run + m->run_off[r], n, r);
  }
  CH_LAUNCHED();
  CH_CUDA(cudaMemcpyAsync(m->run_off_d, m->run_off.data(), sizeof(int) * (R + 1), cudaMemcpyHostToDevice, st));
  if (d == 2) {
    k_elem_vol<2><<<blocks_for(m->E), TPB, 0, st>>>(m->coords, m->elems, m->E, m->vol);
    k_facet_vol<2><<<blocks_for(m->Fb), TPB, 0, st>>>(m->coords, m->bot, m->Fb, m->bvol);
    k_facet_vol<2><<<blocks_for(m->Ft), TPB, 0, st>>>(m->coords, m->top, m->Ft, m->tvol);
  } else {
    k_elem_vol<3><<<blocks_for(m->E), TPB, 0, st>>>(m->coords, m->elems, m->E, m->vol);
    k_facet_vol<3><<<blocks_for(m->Fb), TPB, 0, st>>>(m->coords, m->bot, m->Fb, m->bvol);
    k_facet_vol<3><<<blocks_for(m->Ft), TPB, 0, st>>>(m->coords, m->top, m->Ft, m->tvol);
  }
  CH_LAUNCHED();
  CH_TRY(build_incidence(m->elems, m->E, d + 1, m->N, &m->n2e_ptr, &m->n2e, st, m->mem));
  CH_TRY(build_incidence(m->bot, m->Fb, d, m->N, &m->n2b_ptr, &m->n2b, st, m->mem));
  CH_TRY(build_incidence(m->top, m->Ft, d, m->N, &m->n2t_ptr, &m->n2t, st, m->mem));
  return CH_OK;
}

// ---------------------------------------------------------------- CSR pattern
constexpr int MAXADJ = 128;  // distinct-or-not vertex entries gathered per node

__device__ int gather_adjacent(const int* el, int k, const int* ptr, const int* list, int v,
                               int* buf, int* overflow) {
  int n = 0;
  for (int q = ptr[v]; q < ptr[v + 1]; ++q) {
    const int e = list[q];
    for (int a = 0; a < k; ++a) {
      if (n < MAXADJ) buf[n++] = el[k * e + a];
      else *overflow = 1;
    }
  }
  // insertion sort + unique
  for (int i = 1; i < n; ++i) {
    const int x = buf[i];
    int j = i - 1;
    while (j >= 0 && buf[j] > x) {
      buf[j + 1] = buf[j];
      --j;
    }
    buf[j + 1] = x;
  }
  int u = 0;
  for (int i = 0; i < n; ++i)
    if (u == 0 || buf[u - 1] != buf[i]) buf[u++] = buf[i];
  return u;
}

__global__ void k_pattern(const int* el, int k, const int* ptr, const int* list, int N,
                          const int* rowptr, int* cnt, int* col, int* overflow) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N) return;
  int buf[MAXADJ];
  const int u = gather_adjacent(el, k, ptr, list, v, buf, overflow);
  if (rowptr == nullptr) {
    cnt[v] = u;
  } else {
    for (int i = 0; i < u; ++i) col[rowptr[v] + i] = buf[i];
  }
}

// ---------------------------------------------------------------- values of M and K
__device__ __forceinline__ int find_col(const int* col, int b, int e, int c) {
  while (b < e) {  // binary search in a sorted row
    const int m = (b + e) >> 1;
    if (col[m] < c) b = m + 1;
    else e = m;
  }
  return b;
}

template <int D>
__global__ void k_assemble(const double* X, const int* el, const int* ptr, const int* list, int N,
                           const int* rowptr, const int* col, double* valM, double* valK,
                           int* diag) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N) return;
  const int rb = rowptr[v], re = rowptr[v + 1];
  for (int q = rb; q < re; ++q) {
    valM[q] = 0.0;
    valK[q] = 0.0;
  }
  diag[v] = find_col(col, rb, re, v);
  constexpr double mscale = 1.0 / ((D + 1) * (D + 2));  // M_e = |T| (1 + delta_ab) / ((d+1)(d+2))
  for (int q = ptr[v]; q < ptr[v + 1]; ++q) {
    const int e = list[q];
    const int* ev = el + (D + 1) * e;
    double g[D + 1][D];
    const double vol = simplex_geo<D>(X, ev, g);
    int a = 0;
    while (ev[a] != v) ++a;
    for (int b = 0; b <= D; ++b) {
      double kab = 0.0;
      for (int c = 0; c < D; ++c) kab = fma(g[a][c], g[b][c], kab);
      const int pos = find_col(col, rb, re, ev[b]);
      if (pos < re && col[pos] == ev[b]) {  // always true: the row pattern holds every neighbour
        valK[pos] += vol * kab;
        valM[pos] += vol * mscale * (a == b ? 2.0 : 1.0);
      }
    }
  }
}

__global__ void k_axpby_vals(const double* x, const double* y, double a, double b, double* z,
                             int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = a * x[i] + b * y[i];
}

// ---------------------------------------------------------------- patterned substrate (Section 4)
// With pattern = 1 the substrate energy density of Eq. (5) carries p_p(x) = 1 on the 1st, 3rd and
// 5th sixth of [0, Lx] and p_nfa(x) = 1 on the others (0 elsewhere).  Its boundary load needs, per
// bottom facet F and species s, W1_i = int_F p_s lambda_i and W2_ai = int_F p_s lambda_a lambda_i.
// p_s is constant between breakpoints, so F is clipped to each sixth [lo, hi] and the pieces are
// integrated exactly with the vertex-value rules for linear u, v on a simplex S of dimension k:
//   int_S u = |S| / (k+1) sum_j u_j,   int_S u v = |S| / ((k+1)(k+2)) (sum_j u_j v_j + sum u sum v).
// A 3D facet (a triangle in the x-z plane y = 0) is clipped by Sutherland-Hodgman against the two
// half-planes and fanned into triangles; a 2D facet is a segment of the x axis.
template <int D>
struct FacetHat {  // the facet's hat functions as affine functions of (x, z)
  double X[D], Z[D], det;
  __device__ void lam(double x, double z, double* l) const {
    if constexpr (D == 2) {
      l[1] = (x - X[0]) / (X[1] - X[0]);
      l[0] = 1.0 - l[1];
    } else {
      const double dx = x - X[0], dz = z - Z[0];
      l[1] = (dx * (Z[2] - Z[0]) - (X[2] - X[0]) * dz) / det;
      l[2] = ((X[1] - X[0]) * dz - dx * (Z[1] - Z[0])) / det;
      l[0] = 1.0 - l[1] - l[2];
    }
  }
};

// Adds the integrals over the simplex with vertices P (k + 1 = D of them, measure meas) to W.
template <int D>
__device__ void add_piece(const FacetHat<D>& F, const double (*P)[2], double meas, double* W1, double* W2) {
  double L[D][D];  // L[j][i] = lambda_i at vertex j of the piece
#pragma unroll
  for (int j = 0; j < D; ++j) F.lam(P[j][0], P[j][1], L[j]);
  const double c1 = meas / D, c2 = meas / (D * (D + 1));
#pragma unroll
  for (int i = 0; i < D; ++i) {
    double si = 0.0;
#pragma unroll
    for (int j = 0; j < D; ++j) si += L[j][i];
    W1[i] += c1 * si;
#pragma unroll
    for (int a = 0; a < D; ++a) {
      double sa = 0.0, sai = 0.0;
#pragma unroll
      for (int j = 0; j < D; ++j) {
        sa += L[j][a];
        sai += L[j][a] * L[j][i];
      }
      W2[a * D + i] += c2 * (sai + sa * si);
    }
  }
}

// Clips the convex polygon (x, z)[n] to the half-plane sgn (x - c) >= 0; returns the new vertex
// count.  Each clip adds at most one vertex (a triangle ends with at most 5); cap bounds the
// output all the same.
__device__ int clip_x(const double (*in)[2], int n, double c, double sgn, double (*out)[2], int cap) {
  int k = 0;
  for (int j = 0; j < n && k + 2 <= cap; ++j) {
    const double* P = in[j];
    const double* Q = in[(j + 1) % n];
    const double dp = sgn * (P[0] - c), dq = sgn * (Q[0] - c);
    if (dp >= 0.0) {
      out[k][0] = P[0];
      out[k][1] = P[1];
      ++k;
    }
    if ((dp >= 0.0) != (dq >= 0.0)) {
      const double t = dp / (dp - dq);
      out[k][0] = c;
      out[k][1] = P[1] + t * (Q[1] - P[1]);
      ++k;
    }
  }
  return k;
}

template <int D>
__global__ void k_facet_pattern(const double* coords, const int* bot, int nf, double Lx, double* bw) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  constexpr int NW = D + D * D;
  const int* fv = bot + D * f;
  FacetHat<D> F;
#pragma unroll
  for (int a = 0; a < D; ++a) {
    F.X[a] = coords[(size_t)D * fv[a]];
    F.Z[a] = (D == 3) ? coords[(size_t)D * fv[a] + 2] : 0.0;
  }
  F.det = 0.0;
  if constexpr (D == 3) F.det = (F.X[1] - F.X[0]) * (F.Z[2] - F.Z[0]) - (F.X[2] - F.X[0]) * (F.Z[1] - F.Z[0]);
  double W[2][NW];
#pragma unroll
  for (int q = 0; q < 2 * NW; ++q) W[q / NW][q % NW] = 0.0;
  for (int k = 0; k < 6; ++k) {
    const double lo = k * (Lx / 6.0), hi = (k + 1) * (Lx / 6.0);
    double* W1 = W[k & 1];  // species 0 (polymer) on k = 0, 2, 4; species 1 (NFA) on k = 1, 3, 5
    double* W2 = W1 + D;
    if constexpr (D == 2) {
      const double xa = fmax(fmin(F.X[0], F.X[1]), lo), xb = fmin(fmax(F.X[0], F.X[1]), hi);
      if (xb <= xa) continue;
      const double P[2][2] = {{xa, 0.0}, {xb, 0.0}};
      add_piece<D>(F, P, xb - xa, W1, W2);
    } else {
      double A[8][2], B[8][2];
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        A[a][0] = F.X[a];
        A[a][1] = F.Z[a];
      }
      int n = clip_x(A, 3, lo, 1.0, B, 8);
      n = clip_x(B, n, hi, -1.0, A, 8);
      for (int j = 1; j + 1 < n; ++j) {
        const double P[3][2] = {{A[0][0], A[0][1]}, {A[j][0], A[j][1]}, {A[j + 1][0], A[j + 1][1]}};
        const double meas = 0.5 * fabs((P[1][0] - P[0][0]) * (P[2][1] - P[0][1]) -
                                       (P[2][0] - P[0][0]) * (P[1][1] - P[0][1]));
        if (meas > 0.0) add_piece<D>(F, P, meas, W1, W2);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 2 * NW; ++q) bw[(size_t)f * 2 * NW + q] = W[q / NW][q % NW];
}

// Weights of every run's bottom facets (each run's box is [0, Lx_r] in x).
static ch_status substrate_weights(const ch_mesh_s* m, ch_system_s* s, cudaStream_t st) {
  const int d = m->dim, R = (int)m->runs.size();
  CH_TRY(s->mem.get(&s->bw, (size_t)m->Fb * 2 * (d + d * d)));
  int f0 = 0;
  for (int r = 0; r < R; ++r) {
    int n, e, f;
    box_counts(m->runs[r], &n, &e, &f);
    const int* bot = m->bot + (size_t)f0 * d;
    double* bw = s->bw + (size_t)f0 * 2 * (d + d * d);
    if (f > 0) {
      if (d == 2)
        k_facet_pattern<2><<<blocks_for(f), TPB, 0, st>>>(m->coords, bot, f, m->runs[r].Lx, bw);
      else
        k_facet_pattern<3><<<blocks_for(f), TPB, 0, st>>>(m->coords, bot, f, m->runs[r].Lx, bw);
    }
    f0 += f;
  }
  CH_LAUNCHED();
  return CH_OK;
}

ch_status assemble_system(const ch_mesh_s* m, ch_system_s* s, cudaStream_t st) {
  const int N = m->N, d = m->dim;
  s->N = N;
  Alloc tmp;
  int *cnt = nullptr, *overflow = nullptr;
  CH_TRY(tmp.get(&cnt, (size_t)N));
  CH_TRY(tmp.get(&overflow, 1));
  CH_CUDA(cudaMemsetAsync(overflow, 0, sizeof(int), st));
  k_pattern<<<blocks_for(N), TPB, 0, st>>>(m->elems, d + 1, m->n2e_ptr, m->n2e, N, nullptr, cnt,
                                            nullptr, overflow);
  CH_LAUNCHED();
  CH_TRY(s->mem.get(&s->rowptr, (size_t)N + 1));
  int64_t nnz = 0;
  CH_TRY(scan_i32_to_rowptr(cnt, s->rowptr, N, &nnz, st, tmp));
  s->nnz = nnz;
  CH_TRY(s->mem.get(&s->col, (size_t)nnz));
  CH_TRY(s->mem.get(&s->valM, (size_t)nnz));
  CH_TRY(s->mem.get(&s->valK, (size_t)nnz));
  CH_TRY(s->mem.get(&s->valH, (size_t)nnz));
  CH_TRY(s->mem.get(&s->eload, (size_t)m->E * (d + 1) * 2));
  CH_TRY(s->mem.get(&s->diag, (size_t)N));
  k_pattern<<<blocks_for(N), TPB, 0, st>>>(m->elems, d + 1, m->n2e_ptr, m->n2e, N, s->rowptr,
                                            nullptr, s->col, overflow);
  CH_LAUNCHED();
  if (d == 2)
    k_assemble<2><<<blocks_for(N), TPB, 0, st>>>(m->coords, m->elems, m->n2e_ptr, m->n2e, N,
                                                  s->rowptr, s->col, s->valM, s->valK, s->diag);
  else
    k_assemble<3><<<blocks_for(N), TPB, 0, st>>>(m->coords, m->elems, m->n2e_ptr, m->n2e, N,
                                                  s->rowptr, s->col, s->valM, s->valK, s->diag);
  CH_LAUNCHED();
  // H = a K + sqrt(c) M  (Section 3, matching Schur approximation)
  k_axpby_vals<<<blocks_for(nnz), TPB, 0, st>>>(s->valK, s->valM, s->a, sqrt(s->c), s->valH, nnz);
  CH_LAUNCHED();
  if (s->p.pattern && s->p.bc_mode) CH_TRY(substrate_weights(m, s, st));
  int ovf = 0;
  CH_CUDA(cudaMemcpyAsync(&ovf, overflow, sizeof(int), cudaMemcpyDeviceToHost, st));
  CH_CUDA(cudaStreamSynchronize(st));
  if (ovf) {
    set_error("a node has more than %d incident simplex vertices", MAXADJ);
    return CH_ERR_INTERNAL;
  }
  return CH_OK;
}

// ---------------------------------------------------------------- explicit loads
// Exact integrals of products of linear functions over a simplex T of dimension d:
//   int_T l_1 ... l_n = d! |T| / (d+n)! * sum over permutations pi of {1..n} of
//                       prod over the cycles C of pi of sum_vertices prod_{k in C} l_k(v),
// which follows from int lambda^alpha = d! alpha! |T| / (d+|alpha|)! because alpha! counts
// the permutations fixing an index tuple.  With l = (p, q, q, lambda_i) it gives
//   int p q^2 lambda_i = d!|T|/(d+4)! [ <p><q>^2 + 2<pq><q> + <q^2><p> + 2<pq^2>
//        + p_i(<q>^2 + <q^2>) + 2 q_i(<p><q> + <pq>) + 4 p_i q_i <q> + 2 q_i^2 <p> + 6 p_i q_i^2 ],
// and with (a, b, lambda_i) on a facet of dimension d-1
//   int a b lambda_i = (d-1)!|F|/(d+2)! [ <a><b> + <ab> + a_i<b> + b_i<a> + 2 a_i b_i ],
// where <x> is the sum of x over the simplex's vertices.

struct MeshPod {
  int dim, N, E;
  const double* coords;
  const int* elems;
  const int* bot;
  const int* top;
  const double* vol;
  const double* bvol;
  const double* tvol;
  const int *n2e_ptr, *n2e, *n2b_ptr, *n2b, *n2t_ptr, *n2t;
};

static MeshPod mesh_pod(const ch_mesh_s* s) {
  MeshPod v;
  v.dim = s->dim;
  v.N = s->N;
  v.E = s->E;
  v.coords = s->coords;
  v.elems = s->elems;
  v.bot = s->bot;
  v.top = s->top;
  v.vol = s->vol;
  v.bvol = s->bvol;
  v.tvol = s->tvol;
  v.n2e_ptr = s->n2e_ptr;
  v.n2e = s->n2e;
  v.n2b_ptr = s->n2b_ptr;
  v.n2b = s->n2b;
  v.n2t_ptr = s->n2t_ptr;
  v.n2t = s->n2t;
  return v;
}

struct LoadCoef {
  double cs;      // coefficient of phi_s in f' (0.2 for Eq. (15), 0 otherwise)
  double cubic;   // 7 for Eq. (15), 0 for f' = 0
  int bc;         // boundary loads on/off
  double gp, gn, hp, hn, kev;
  const double* bw;  // patterned substrate weights (Fb x 2 x (D + D^2)), or null for p = 1
};

// Per element e and vertex a, eload[(e (D+1) + a) 2 + {0, 1}] = |T| (7 int p q^2 l_a - 0.2 int phi_s l_a)
// / |T| and the same with p and q exchanged (Eq. (15)'s f' for polymer and NFA against the hat
// function of vertex a).  The vertex sums are formed once per element; int_pqq_li's terms that do
// not involve the vertex (A, B, C below) are element constants (the closed form above).
template <int D>
__global__ void k_elem_loads(const MeshPod m, LoadCoef L, const double* pp, const double* pn, int ld,
                             double* __restrict__ eload) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.E) return;
  constexpr double c4 = (D == 2) ? 1.0 / 360.0 : 1.0 / 840.0;  // d!/(d+4)!
  constexpr double c2 = 1.0 / ((D + 1) * (D + 2));             // int lambda_a lambda_i / |T|, a != i
  const int* ev = m.elems + (D + 1) * e;
  double P[D + 1], Q[D + 1];
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    P[a] = pp[(size_t)ld * ev[a]];
    Q[a] = pn[(size_t)ld * ev[a]];
  }
  double Sp = 0, Sq = 0, Spq = 0, Spp = 0, Sqq = 0, Spqq = 0, Sppq = 0;
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    Sp += P[a];
    Sq += Q[a];
    const double pq = P[a] * Q[a];
    Spq += pq;
    Spp += P[a] * P[a];
    Sqq += Q[a] * Q[a];
    Spqq += pq * Q[a];
    Sppq += pq * P[a];
  }
  // int p q^2 l_i / (c4 |T|) = A + p_i B + q_i (C + 2 q_i Sp) + p_i q_i (4 Sq + 6 q_i), and the
  // same with p and q exchanged (C is symmetric)
  const double Ap = Sp * Sq * Sq + 2.0 * Spq * Sq + Sqq * Sp + 2.0 * Spqq, Bp = Sq * Sq + Sqq;
  const double An = Sq * Sp * Sp + 2.0 * Spq * Sp + Spp * Sq + 2.0 * Sppq, Bn = Sp * Sp + Spp;
  const double C = 2.0 * (Sp * Sq + Spq);
  const double vol = m.vol[e];
  const double ss = (D + 1) - Sp - Sq;  // sum of phi_s over the vertices
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    const double pi = P[a], qi = Q[a];
    const double Ip = c4 * (Ap + pi * Bp + qi * (C + 2.0 * qi * Sp) + pi * qi * (4.0 * Sq + 6.0 * qi));
    const double In = c4 * (An + qi * Bn + pi * (C + 2.0 * pi * Sq) + qi * pi * (4.0 * Sp + 6.0 * pi));
    const double Is = c2 * (ss + (1.0 - pi - qi));  // int phi_s lambda_i / |T|
    double2 out;
    out.x = vol * (L.cubic * Ip - L.cs * Is);
    out.y = vol * (L.cubic * In - L.cs * Is);
    reinterpret_cast<double2*>(eload)[(size_t)e * (D + 1) + a] = out;
  }
}

// ---- The Flory-Huggins load (potential = 3).  Section 2's bulk energy
//   f = phi_p ln(phi_p) / N_p + phi_n ln(phi_n) / N_n + phi_s ln(phi_s) / N_s
//       + chi_pn phi_p phi_n + chi_ps phi_p phi_s + chi_ns phi_n phi_s,   phi_s = 1 - phi_p - phi_n,
// differentiated through phi_s like Eq. (15):
//   f_p' = (ln phi_p + 1) / N_p - (ln phi_s + 1) / N_s + chi_pn phi_n + chi_ps (phi_s - phi_p) - chi_ns phi_n
//   f_n' = (ln phi_n + 1) / N_n - (ln phi_s + 1) / N_s + (chi_pn - chi_ps) phi_p + chi_ns (phi_s - phi_n)
// with each logarithm taken at max(phi, delta) (a NaN stays a NaN).  The integrand is not a
// polynomial, so a fixed rule defines the load: on every simplex the product of 3-point
// Gauss-Legendre rules collapsed onto it (Duffy), 9 points on a triangle, 27 on a tetrahedron.
struct FhRule {
  int nq;
  double lam[27][4];  // barycentric coordinates of the points
  double w[27];       // weights, summing to 1: int_T g ~ |T| sum_q w_q g(x_q)
};

struct FhCoef {
  double chi_pn, chi_ps, chi_ns, inv_np, inv_nn, inv_ns, delta;
};

// Gauss-Legendre on [0, 1] with 3 points: 1/2 -+ sqrt(15)/10 and 1/2, weights 5/18, 4/9, 5/18.
// Square (u, v) -> triangle (u, v (1 - u)), Jacobian 1 - u; cube (u, v, t) -> tetrahedron
// (u, v (1 - u), t (1 - u)(1 - v)), Jacobian (1 - u)^2 (1 - v); normalised by the reference
// simplex's measure (1/2, 1/6).
static FhRule fh_rule(int dim) {
  const double g[3] = {0.5 - std::sqrt(15.0) / 10.0, 0.5, 0.5 + std::sqrt(15.0) / 10.0};
  const double w[3] = {5.0 / 18.0, 4.0 / 9.0, 5.0 / 18.0};
  FhRule R{};
  int q = 0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < (dim == 3 ? 3 : 1); ++k) {
        const double u = g[i], v = g[j];
        double xi[3] = {u, v * (1.0 - u), 0.0};
        double wt;
        if (dim == 2) {
          wt = 2.0 * w[i] * w[j] * (1.0 - u);
        } else {
          xi[2] = g[k] * (1.0 - u) * (1.0 - v);
          wt = 6.0 * w[i] * w[j] * w[k] * (1.0 - u) * (1.0 - u) * (1.0 - v);
        }
        R.lam[q][0] = 1.0 - xi[0] - xi[1] - xi[2];
        for (int a = 1; a <= dim; ++a) R.lam[q][a] = xi[a - 1];
        R.w[q] = wt;
        ++q;
      }
  R.nq = q;
  return R;
}

__device__ __forceinline__ double guarded_log(double x, double delta) { return log(x < delta ? delta : x); }

// eload[(e (D+1) + a) 2 + {0, 1}] = |T| sum_q w_q f_{p,n}'(phi_h(x_q)) lambda_a(x_q)
template <int D>
__global__ void k_elem_loads_fh(const MeshPod m, const FhRule R, const FhCoef F, const double* pp,
                                const double* pn, int ld, double* __restrict__ eload) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m.E) return;
  const int* ev = m.elems + (D + 1) * e;
  double P[D + 1], Q[D + 1], Fp[D + 1], Fn[D + 1];
#pragma unroll
  for (int a = 0; a <= D; ++a) {
    P[a] = pp[(size_t)ld * ev[a]];
    Q[a] = pn[(size_t)ld * ev[a]];
    Fp[a] = 0.0;
    Fn[a] = 0.0;
  }
  for (int q = 0; q < R.nq; ++q) {
    double p = 0.0, n = 0.0;
#pragma unroll
    for (int a = 0; a <= D; ++a) {
      p += R.lam[q][a] * P[a];
      n += R.lam[q][a] * Q[a];
    }
    const double s = 1.0 - p - n;
    const double ls = (guarded_log(s, F.delta) + 1.0) * F.inv_ns;
    const double fp = (guarded_log(p, F.delta) + 1.0) * F.inv_np - ls + F.chi_pn * n + F.chi_ps * (s - p) -
                      F.chi_ns * n;
    const double fn = (guarded_log(n, F.delta) + 1.0) * F.inv_nn - ls + (F.chi_pn - F.chi_ps) * p +
                      F.chi_ns * (s - n);
    const double wq = R.w[q];
#pragma unroll
    for (int a = 0; a <= D; ++a) {
      Fp[a] += wq * fp * R.lam[q][a];
      Fn[a] += wq * fn * R.lam[q][a];
    }
  }
  const double vol = m.vol[e];
#pragma unroll
  for (int a = 0; a <= D; ++a)
    reinterpret_cast<double2*>(eload)[(size_t)e * (D + 1) + a] = make_double2(vol * Fp[a], vol * Fn[a]);
}

template <int D>
__device__ void node_loads(const MeshPod& m, const LoadCoef& L, const double* __restrict__ eload,
                           const double* pp, const double* pn, int ld, int v, double* Fp, double* Fn,
                           double* Gp, double* Gn) {
  double fp = 0.0, fn = 0.0;
  for (int q = m.n2e_ptr[v]; q < m.n2e_ptr[v + 1]; ++q) {  // incident elements in a fixed order
    const int e = m.n2e[q];
    const int* ev = m.elems + (D + 1) * e;
    int li = 0;
#pragma unroll
    for (int a = 0; a <= D; ++a)
      if (ev[a] == v) li = a;
    const double2 c = reinterpret_cast<const double2*>(eload)[(size_t)e * (D + 1) + li];
    fp += c.x;
    fn += c.y;
  }
  *Fp = fp;
  *Fn = fn;
  double gp = 0.0, gn = 0.0;
  if (L.bc) {
    constexpr int DF = D - 1;
    constexpr double f1 = 1.0 / (DF + 1);                 // int lambda_i / |F|
    constexpr double f2 = 1.0 / ((DF + 1) * (DF + 2));    // int lambda_a lambda_i / |F|, a != i
    constexpr double f3 = (D == 2) ? 1.0 / 24.0 : 1.0 / 60.0;  // (d-1)!/(d+2)!
    if (L.bw) {
      // Gamma_b, patterned: int p_s (g + 2 h phi) lambda_i = g W1_i + 2 h sum_a phi_a W2_ai
      for (int q = m.n2b_ptr[v]; q < m.n2b_ptr[v + 1]; ++q) {
        const int f = m.n2b[q];
        const int* fv = m.bot + D * f;
        const double* Wp = L.bw + (size_t)f * 2 * (D + D * D);
        const double* Wn = Wp + D + D * D;
        int li = 0;
        for (int a = 0; a < D; ++a)
          if (fv[a] == v) li = a;
        double sp = 0.0, sn = 0.0;
        for (int a = 0; a < D; ++a) {
          sp += pp[(size_t)ld * fv[a]] * Wp[D + a * D + li];
          sn += pn[(size_t)ld * fv[a]] * Wn[D + a * D + li];
        }
        gp += L.gp * Wp[li] + 2.0 * L.hp * sp;
        gn += L.gn * Wn[li] + 2.0 * L.hn * sn;
      }
    } else {
      for (int q = m.n2b_ptr[v]; q < m.n2b_ptr[v + 1]; ++q) {  // Gamma_b: int (g + 2 h phi) lambda_i
        const int f = m.n2b[q];
        const int* fv = m.bot + D * f;
        double Sp = 0, Sq = 0, pi = 0, qi = 0;
        for (int a = 0; a < D; ++a) {
          Sp += pp[(size_t)ld * fv[a]];
          Sq += pn[(size_t)ld * fv[a]];
          if (fv[a] == v) {
            pi = pp[(size_t)ld * fv[a]];
            qi = pn[(size_t)ld * fv[a]];
          }
        }
        const double ar = m.bvol[f];
        gp += ar * (L.gp * f1 + 2.0 * L.hp * f2 * (Sp + pi));
        gn += ar * (L.gn * f1 + 2.0 * L.hn * f2 * (Sq + qi));
      }
    }
    for (int q = m.n2t_ptr[v]; q < m.n2t_ptr[v + 1]; ++q) {  // Gamma_t: k int phi phi_s lambda_i
      const int f = m.n2t[q];
      const int* fv = m.top + D * f;
      double Sp = 0, Sq = 0, Ss = 0, Sps = 0, Sqs = 0, pi = 0, qi = 0, si = 0;
      for (int a = 0; a < D; ++a) {
        const double x = pp[(size_t)ld * fv[a]], y = pn[(size_t)ld * fv[a]], s = 1.0 - x - y;
        Sp += x;
        Sq += y;
        Ss += s;
        Sps += x * s;
        Sqs += y * s;
        if (fv[a] == v) {
          pi = x;
          qi = y;
          si = s;
        }
      }
      const double ar = m.tvol[f] * L.kev * f3;
      gp += ar * (Sp * Ss + Sps + pi * Ss + si * Sp + 2.0 * pi * si);
      gn += ar * (Sq * Ss + Sqs + qi * Ss + si * Sq + 2.0 * qi * si);
    }
  }
  *Gp = gp;
  *Gn = gn;
}

static LoadCoef load_coef(const ch_params& p) {
  LoadCoef L;
  L.cubic = p.potential == 2 ? 0.0 : 7.0;
  L.cs = p.potential == 0 ? 0.2 : 0.0;
  L.bc = p.bc_mode;
  L.gp = p.g_p;
  L.gn = p.g_nfa;
  L.hp = p.h_p;
  L.hn = p.h_nfa;
  L.kev = p.evap_sign * p.k_evap;
  L.bw = nullptr;
  return L;
}

template <int D>
__global__ void k_loads(const MeshPod m, LoadCoef L, const double* eload, const double* pp,
                        const double* pn, int ld, double* Fp, double* Fn, double* Gp, double* Gn) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= m.N) return;
  double a, b, c, d;
  node_loads<D>(m, L, eload, pp, pn, ld, v, &a, &b, &c, &d);
  if (Fp) Fp[v] = a;
  if (Fn) Fn[v] = b;
  if (Gp) Gp[v] = c;
  if (Gn) Gn[v] = d;
}

// b (N x 4) = (M phi_p + tau g_p, M phi_n + tau g_n, -c F_p, -c F_n)   (Eq. (13) -> Eq. (14))
template <int D>
__global__ void k_rhs(const MeshPod m, LoadCoef L, const double* eload, const int* rowptr,
                      const int* col, const double* valM, const double* pp, const double* pn, int ld,
                      double tau, double c, double* b) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= m.N) return;
  double Fp, Fn, Gp, Gn;
  node_loads<D>(m, L, eload, pp, pn, ld, v, &Fp, &Fn, &Gp, &Gn);
  double mp = 0.0, mn = 0.0;
  for (int q = rowptr[v]; q < rowptr[v + 1]; ++q) {
    const int j = col[q];
    mp = fma(valM[q], pp[(size_t)ld * j], mp);
    mn = fma(valM[q], pn[(size_t)ld * j], mn);
  }
  double4_32a out;
  out.x = mp + tau * Gp;
  out.y = mn + tau * Gn;
  out.z = -c * Fp;
  out.w = -c * Fn;
  reinterpret_cast<double4_32a*>(b)[v] = out;
}

// Per-element load contributions into s->eload (the system's scratch: calls on one system must
// not overlap on the GPU).  Algorithmic bytes: the vertex values gathered, element indices and
// measures, the contributions written.
static void elem_loads(const ch_system_s* s, const MeshPod& m, const LoadCoef& L, const double* pp,
                       const double* pn, int ld, cudaStream_t st) {
  const double E = m.E, d1 = m.dim + 1;
  if (s->p.potential == 3) {
    const FhRule R = fh_rule(m.dim);
    const ch_params& p = s->p;
    const FhCoef F{p.chi_pn, p.chi_ps, p.chi_ns, 1.0 / p.N_p, 1.0 / p.N_nfa, 1.0 / p.N_s, p.fh_delta};
    ProfScope ps(st, K_ELEM_LOADS, 0, E * (d1 * (4.0 + 16.0) + 8.0 + 16.0 * d1), E * R.nq * (4.0 * d1 + 10.0));
    if (m.dim == 2)
      k_elem_loads_fh<2><<<blocks_for(m.E), TPB, 0, st>>>(m, R, F, pp, pn, ld, s->eload);
    else
      k_elem_loads_fh<3><<<blocks_for(m.E), TPB, 0, st>>>(m, R, F, pp, pn, ld, s->eload);
    return;
  }
  ProfScope ps(st, K_ELEM_LOADS, 0, E * (d1 * (4.0 + 16.0) + 8.0 + 16.0 * d1), E * (22.0 + 12.0 * d1));
  if (m.dim == 2)
    k_elem_loads<2><<<blocks_for(m.E), TPB, 0, st>>>(m, L, pp, pn, ld, s->eload);
  else
    k_elem_loads<3><<<blocks_for(m.E), TPB, 0, st>>>(m, L, pp, pn, ld, s->eload);
}

ch_status loads(const ch_system_s* s, const double* pp, const double* pn, double* Fp, double* Fn,
                double* gp, double* gn, cudaStream_t st) {
  const MeshPod m = mesh_pod(s->mesh);
  LoadCoef L = load_coef(s->p);
  L.bw = s->bw;
  elem_loads(s, m, L, pp, pn, 1, st);
  ProfScope ps(st, K_LOADS, 0, 16.0 * m.N + 32.0 * m.N, 0.0);
  if (m.dim == 2)
    k_loads<2><<<blocks_for(m.N), TPB, 0, st>>>(m, L, s->eload, pp, pn, 1, Fp, Fn, gp, gn);
  else
    k_loads<3><<<blocks_for(m.N), TPB, 0, st>>>(m, L, s->eload, pp, pn, 1, Fp, Fn, gp, gn);
  CH_LAUNCHED();
  return CH_OK;
}

ch_status rhs_strided(const ch_system_s* s, const double* pp, const double* pn, int ld, double* b,
                      cudaStream_t st) {
  const MeshPod m = mesh_pod(s->mesh);
  LoadCoef L = load_coef(s->p);
  L.bw = s->bw;
  elem_loads(s, m, L, pp, pn, ld, st);
  const double E = s->mesh->E, d1 = m.dim + 1;
  // phi read + b written + M (values, columns, row pointers) + incidence and the element
  // contributions gathered
  ProfScope ps(st, K_RHS, 0, 48.0 * m.N + 12.0 * s->nnz + 4.0 * m.N + E * d1 * (4.0 + 4.0 + 16.0),
               2.0 * s->nnz);
  if (m.dim == 2)
    k_rhs<2><<<blocks_for(m.N), TPB, 0, st>>>(m, L, s->eload, s->rowptr, s->col, s->valM, pp, pn, ld,
                                               s->p.tau, s->c, b);
  else
    k_rhs<3><<<blocks_for(m.N), TPB, 0, st>>>(m, L, s->eload, s->rowptr, s->col, s->valM, pp, pn, ld,
                                               s->p.tau, s->c, b);
  CH_LAUNCHED();
  return CH_OK;
}

// ---------------------------------------------------------------- block operator of Eq. (14)
// y = A x for both species: per node x = (x1_p, x1_n, x2_p, x2_n),
//   y1 = M x1 + a K x2,  y2 = a K x1 - c M x2.
// One pass over the shared pattern: 8 FMAs per stored entry.
__global__ void k_apply_A(int N, const int* rowptr, const int* col, const double* valM,
                          const double* valK, double a, double c, const double4_32a* x, double4_32a* y) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= N) return;
  double m1p = 0, m1n = 0, m2p = 0, m2n = 0, k1p = 0, k1n = 0, k2p = 0, k2n = 0;
  for (int q = rowptr[v]; q < rowptr[v + 1]; ++q) {
    const int j = col[q];
    const double m = valM[q], k = valK[q];
    const double4_32a z = x[j];
    m1p = fma(m, z.x, m1p);
    m1n = fma(m, z.y, m1n);
    m2p = fma(m, z.z, m2p);
    m2n = fma(m, z.w, m2n);
    k1p = fma(k, z.x, k1p);
    k1n = fma(k, z.y, k1n);
    k2p = fma(k, z.z, k2p);
    k2n = fma(k, z.w, k2n);
  }
  double4_32a out;
  out.x = fma(a, k2p, m1p);
  out.y = fma(a, k2n, m1n);
  out.z = fma(a, k1p, -c * m2p);
  out.w = fma(a, k1n, -c * m2n);
  y[v] = out;
}

ch_status apply_A(const ch_system_s* s, const double* x, double* y, cudaStream_t st) {
  ProfScope ps(st, K_APPLY_A, 0, 20.0 * s->nnz + 4.0 * (s->N + 1) + 64.0 * s->N,
               8.0 * s->nnz + 4.0 * s->N);
  k_apply_A<<<blocks_for(s->N), TPB, 0, st>>>(s->N, s->rowptr, s->col, s->valM, s->valK, s->a,
                                               s->c, reinterpret_cast<const double4_32a*>(x),
                                               reinterpret_cast<double4_32a*>(y));
  CH_LAUNCHED();
  return CH_OK;
}

}  // namespace ch
