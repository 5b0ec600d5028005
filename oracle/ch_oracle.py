"""Plain FP64 CPU oracle of the per-time-step solve of the ternary Cahn-Hilliard model.

TEST INFRASTRUCTURE ONLY.  This module exists to check the CUDA library.  Only
the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import or run it; the library itself never does, and
it shares no code with the CUDA sources.

Everything here is written out from the paper's statement of the method in
plain numpy / scipy, in float64, with no blocking or fusion:

* mesh           -- uniform simplicial meshes of a box (Section 4, first paragraph)
* element_matrices / assemble -- P1 mass M and stiffness K (Section 3, below Eq. (12))
* load_vector    -- f^(k): the exact load of df/dphi for the polynomial
                    potential Eq. (15), explicit in time (Section 3, Eq. (12))
* boundary_load  -- the flux boundary conditions Eq. (10) on Gamma_b and Gamma_t
* saddle_matrix / rhs -- the symmetric saddle-point system Eq. (14)
* Solver.step    -- one semi-implicit step Eq. (12)/(13): the exact solution of
                    Eq. (14) for both species by a direct factorisation
* schur / schur_tilde -- S and its matching approximation (Section 3, Lemma 1)
* chebyshev_semi_iteration -- M~ by the Chebyshev semi-iteration Section 3 names as the
                    alternative to AMG (Jacobi-preconditioned, Wathen's eigenvalue bounds)
* flory_huggins / dfdphi_fh / load_vector_fh -- the logarithmic bulk energy of Section 2
                    and its load (reading R14)
* chebyshev_smooth / vcycle / galerkin_levels -- one multigrid V-cycle over a given
                    hierarchy (Chebyshev smoothing, P^T restriction, exact coarsest solve): the
                    inner solves of Algorithm 1 written from their definition

Readings of points the paper leaves open:
  R1 the discrete coefficient of K phi in the mu equation is eps (Eq. (12)/(14)),
     not eps^2 as in the strong form Eq. (9);
  R2 mobilities are 1 unless given ("appropriate constants");
  R3 df/dphi_p differentiates f(phi_p, phi_nfa, 1 - phi_p - phi_nfa) by the chain
     rule: f_p' = 7 phi_p phi_nfa^2 - 0.2 phi_s ('poly'); 'poly_partial' drops the
     solvent term, 'none' sets f' = 0 (used by closed-form tests), 'fh' is the
     Flory-Huggins f of R14;
  R4 f^(k) is the exact load vector int f'(phi_h^k) lambda_i, not M f'(phi^k);
  R5 the evaporation flux on Gamma_t enters with sign ``evap_sign`` (+1: inflow of
     polymer and NFA as the text describes; -1: Eq. (10) read literally);
  R6 the substrate flux on Gamma_b is +df_s/dphi (Eq. (10) literally), with
     p_p = p_nfa = 1, or with ``pattern`` = 1 Section 4's alternating preference:
     p_p = 1 on the 1st, 3rd and 5th sixth of [0, Lx], p_nfa = 1 on the others
     (the shared endpoints of the closed subintervals have measure zero);
  R7 no extra boundary term in the mu equation (natural condition grad phi . n = 0);
  R8 2D cells split along the lower-left/upper-right diagonal, 3D hexahedra into
     the 6 Kuhn tetrahedra; Gamma_b = {y = 0}, Gamma_t = {y = L_y}.
  R14 the Flory-Huggins f (Section 2) is differentiated through phi_s like Eq. (15)
     (R3), with Section 4's chi and N; its logarithms are evaluated at max(phi, delta)
     (the positivity guard the paper's polynomial replacement avoids needing); its load
     is defined by the collapsed 3-point Gauss-Legendre rule on each simplex, the
     integrand not being a polynomial.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

DENSE_LIMIT = 6000  # 2N at or below this: dense LU; above: sparse LU


@dataclass
class Params:
    """Model and discretisation parameters; defaults are the paper's (Section 4)."""
    dim: int = 2
    nx: int = 32
    ny: int = 32
    nz: int = 0
    Lx: float = 1.0
    Ly: float = 1.0
    Lz: float = 1.0
    tau: float = 1e-4          # scaled time step (Fig. 1 caption)
    eps: float = 1e-3          # eps_p = eps_nfa (Section 4)
    mobility: float = 1.0      # reading R2
    bc_mode: int = 1           # 0: zero flux everywhere, 1: fluxes of Eq. (10)
    k_evap: float = 5e-3       # evaporation rate k (Section 4)
    evap_sign: int = 1         # reading R5
    g_p: float = 0.01          # substrate parameters g, h of Eq. (5) (Section 4)
    g_nfa: float = 0.01
    h_p: float = 0.0
    h_nfa: float = 0.0
    potential: str = "poly"    # reading R3
    pattern: int = 0           # substrate patterning p_p(x), p_nfa(x) of Section 4 (reading R6)
    chi_pn: float = 1.0        # Flory-Huggins interaction parameters (Section 4)
    chi_ps: float = 0.3
    chi_ns: float = 0.3
    N_p: float = 20.0          # degrees of polymerisation (Section 4)
    N_nfa: float = 20.0
    N_s: float = 1.0
    fh_delta: float = 1e-10    # positivity guard: each logarithm at max(phi, fh_delta)


# ----------------------------------------------------------------------------
# Mesh (Section 4: uniform triangulations of a box; reading R8)
# ----------------------------------------------------------------------------
@dataclass
class Mesh:
    dim: int
    coords: np.ndarray        # (N, d) float64
    elems: np.ndarray         # (E, d+1) int64
    bottom: np.ndarray        # (Fb, d) facets on y = 0
    top: np.ndarray           # (Ft, d) facets on y = Ly
    ijk: np.ndarray = field(repr=False, default=None)  # (N, d) integer grid index


def mesh(p: Params) -> Mesh:
    """Uniform P1 mesh of [0,Lx]x[0,Ly](x[0,Lz]); node index i + (nx+1)(j + (ny+1)k)."""
    if p.dim == 2:
        nx, ny = p.nx, p.ny
        j, i = np.meshgrid(np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
        ijk = np.c_[i.ravel(), j.ravel()]
        coords = np.c_[ijk[:, 0] * (p.Lx / nx), ijk[:, 1] * (p.Ly / ny)]
        cj, ci = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
        v00 = (ci + (nx + 1) * cj).ravel()
        v10, v01 = v00 + 1, v00 + nx + 1
        v11 = v01 + 1
        # cell c -> elements 2c (v00,v10,v11) and 2c+1 (v00,v11,v01)
        elems = np.stack([np.c_[v00, v10, v11], np.c_[v00, v11, v01]], 1).reshape(-1, 3)
    elif p.dim == 3:
        nx, ny, nz = p.nx, p.ny, p.nz
        k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
        ijk = np.c_[i.ravel(), j.ravel(), k.ravel()]
        coords = np.c_[ijk[:, 0] * (p.Lx / nx), ijk[:, 1] * (p.Ly / ny), ijk[:, 2] * (p.Lz / nz)]
        ck, cj, ci = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
        ci, cj, ck = ci.ravel(), cj.ravel(), ck.ravel()

        def node(off):
            return (ci + off[0]) + (nx + 1) * ((cj + off[1]) + (ny + 1) * (ck + off[2]))

        tets = []
        for perm in itertools.permutations(range(3)):   # Kuhn: v000 -> +e_a -> +e_b -> v111
            off = [0, 0, 0]
            verts = [node(off)]
            for a in perm:
                off[a] = 1
                verts.append(node(off))
            tets.append(np.stack(verts, 1))
        elems = np.stack(tets, 1).reshape(-1, 4)
    else:
        raise ValueError("dim must be 2 or 3")
    # boundary facets: element faces whose vertices all lie on y = 0 (resp. y = Ly)
    d = p.dim
    faces = np.concatenate([np.delete(elems, a, axis=1) for a in range(d + 1)])
    jy = ijk[:, 1][faces]
    bottom = faces[(jy == 0).all(1)]
    top = faces[(jy == p.ny).all(1)]
    return Mesh(d, coords.astype(np.float64), elems.astype(np.int64), bottom, top, ijk)


# ----------------------------------------------------------------------------
# P1 element matrices and assembly (Section 3: "standard mass and stiffness matrices")
# ----------------------------------------------------------------------------
def simplex_measure_and_gradients(X: np.ndarray):
    """|T| and the gradients of the barycentric coordinates, per simplex.

    X: (E, d+1, d) vertex coordinates.  lambda_{1..d}(x) = J^{-1}(x - x_0) with
    J = [x_1 - x_0, ..., x_d - x_0], so grad lambda_k is row k of J^{-1} and
    grad lambda_0 = -sum_k grad lambda_k.
    """
    d = X.shape[2]
    J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))
    vol = np.abs(np.linalg.det(J)) / math.factorial(d)
    Jinv = np.linalg.inv(J)
    G = np.concatenate([-Jinv.sum(axis=1, keepdims=True), Jinv], axis=1)  # (E, d+1, d)
    return vol, G


def element_matrices(X: np.ndarray):
    """M_e = |T|(1 + delta_ab)/((d+1)(d+2)),  K_e = |T| grad lambda_a . grad lambda_b."""
    d = X.shape[2]
    vol, G = simplex_measure_and_gradients(X)
    Ke = vol[:, None, None] * np.einsum("ead,ebd->eab", G, G)
    base = (np.ones((d + 1, d + 1)) + np.eye(d + 1)) / ((d + 1) * (d + 2))
    Me = vol[:, None, None] * base[None]
    return Me, Ke


def assemble(m: Mesh):
    """Global CSR M and K (sum over elements of the scattered element matrices)."""
    N = m.coords.shape[0]
    Me, Ke = element_matrices(m.coords[m.elems])
    n = m.dim + 1
    rows = np.repeat(m.elems, n, axis=1).ravel()
    cols = np.tile(m.elems, (1, n)).ravel()
    M = sp.csr_matrix((Me.ravel(), (rows, cols)), shape=(N, N))
    K = sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(N, N))
    for A in (M, K):
        A.sum_duplicates()
        A.sort_indices()
    return M, K


# ----------------------------------------------------------------------------
# Exact integrals of barycentric monomials: int_T lambda^alpha = d! alpha! |T| / (d + |alpha|)!
# ----------------------------------------------------------------------------
def monomial_table(d: int, order: int) -> np.ndarray:
    """T[a_1,...,a_order] = (1/|T|) int_T lambda_{a_1} ... lambda_{a_order} on a d-simplex."""
    n = d + 1
    T = np.empty((n,) * order)
    for idx in itertools.product(range(n), repeat=order):
        alpha = np.bincount(np.array(idx, dtype=np.int64), minlength=n)
        num = math.factorial(d) * np.prod([math.factorial(a) for a in alpha])
        T[idx] = num / math.factorial(d + order)
    return T


def dfdphi(pp: np.ndarray, pn: np.ndarray, potential: str):
    """Nodal df/dphi_p, df/dphi_nfa for f = 3.5 phi_p^2 phi_nfa^2 + 0.1 phi_s^2, Eq. (15)."""
    ps = 1.0 - pp - pn
    if potential == "poly":
        return 7.0 * pp * pn ** 2 - 0.2 * ps, 7.0 * pp ** 2 * pn - 0.2 * ps
    if potential == "poly_partial":
        return 7.0 * pp * pn ** 2, 7.0 * pp ** 2 * pn
    if potential == "none":
        return np.zeros_like(pp), np.zeros_like(pn)
    raise ValueError(potential)


def load_vector(m: Mesh, pp: np.ndarray, pn: np.ndarray, potential: str = "poly"):
    """F_s[i] = int_Omega df/dphi_s(phi_h) lambda_i, exactly (reading R4).

    f_p' = 7 phi_p phi_n^2 - c_s (1 - phi_p - phi_n) with c_s = 0.2 ('poly') or 0;
    the integrand is a polynomial of degree 4 in the barycentric coordinates, so
    the monomial formula integrates it exactly.
    """
    d = m.dim
    N = m.coords.shape[0]
    vol, _ = simplex_measure_and_gradients(m.coords[m.elems])
    P, Q = pp[m.elems], pn[m.elems]                       # (E, d+1) vertex values
    if potential == "none":
        return np.zeros(N), np.zeros(N)
    T4, T2, T1 = monomial_table(d, 4), monomial_table(d, 2), monomial_table(d, 1)
    cubic_p = 7.0 * np.einsum("ea,eb,ec,abci->ei", P, Q, Q, T4)   # int phi_p phi_n^2 lambda_i / |T|
    cubic_n = 7.0 * np.einsum("ea,eb,ec,abci->ei", P, P, Q, T4)   # int phi_p^2 phi_n lambda_i / |T|
    if potential == "poly":
        solv = T1[None, :] - np.einsum("ea,ai->ei", P + Q, T2)    # int phi_s lambda_i / |T|
        cubic_p = cubic_p - 0.2 * solv
        cubic_n = cubic_n - 0.2 * solv
    Fp = np.zeros(N)
    Fn = np.zeros(N)
    np.add.at(Fp, m.elems, vol[:, None] * cubic_p)
    np.add.at(Fn, m.elems, vol[:, None] * cubic_n)
    return Fp, Fn


def facet_measure(X: np.ndarray) -> np.ndarray:
    """Length (d=2) or area (d=3) of boundary facets with vertex coordinates X (F, d, d)."""
    if X.shape[1] == 2:
        return np.linalg.norm(X[:, 1] - X[:, 0], axis=1)
    return 0.5 * np.linalg.norm(np.cross(X[:, 1] - X[:, 0], X[:, 2] - X[:, 0]), axis=1)


def substrate_preference(x: np.ndarray, Lx: float):
    """(p_p(x), p_nfa(x)) of Section 4's patterned substrate for points inside [0, Lx]: the
    interval is cut into six equal parts, polymer preferred on the 1st, 3rd and 5th."""
    k = np.clip(np.floor(6.0 * np.asarray(x, dtype=np.float64) / Lx), 0, 5).astype(np.int64)
    pref_p = (k % 2 == 0).astype(np.float64)
    return pref_p, 1.0 - pref_p


GAUSS3 = np.polynomial.legendre.leggauss(3)  # exact for degree 5 on an interval


def _gauss_on(a: float, b: float):
    """3-point Gauss-Legendre nodes and weights on [a, b]."""
    x, w = GAUSS3
    return 0.5 * (a + b) + 0.5 * (b - a) * x, 0.5 * (b - a) * w


def _patterned_substrate(m: Mesh, pp: np.ndarray, pn: np.ndarray, p: Params, gp, gn):
    """Adds int_{Gamma_b} p_s(x) (g_s + 2 h_s phi_s) lambda_i to gp, gn (Eq. (5), Section 4).

    p_s is piecewise constant in x, so each facet is cut at the breakpoints k Lx / 6 that cross
    it (and, in 3D, at its own vertices' x, where the facet's cross-section changes edges).  On
    each piece the integrand is a polynomial of degree <= 2 in the facet's coordinates; nested
    3-point Gauss-Legendre rules (x outside, z inside for a 3D facet) integrate it exactly."""
    breaks = np.arange(1, 6) * (p.Lx / 6.0)
    for f in m.bottom:
        X = m.coords[f]
        if m.dim == 2:
            x0, x1 = X[0, 0], X[1, 0]
            lo, hi = min(x0, x1), max(x0, x1)
            cuts = np.unique(np.r_[lo, hi, breaks[(breaks > lo) & (breaks < hi)]])
            for a, b in zip(cuts[:-1], cuts[1:]):
                xq, wq = _gauss_on(a, b)
                l1 = (xq - x0) / (x1 - x0)
                lam = np.c_[1.0 - l1, l1]                    # (q, 2) hat functions on the facet
                _accumulate(f, lam, wq, xq, pp, pn, p, gp, gn)
        else:
            P = X[:, [0, 2]]                                  # the facet lies in y = 0: (x, z)
            T = np.c_[P[1] - P[0], P[2] - P[0]]               # x-z Jacobian of the facet
            lo, hi = P[:, 0].min(), P[:, 0].max()
            cuts = np.unique(np.r_[P[:, 0], breaks[(breaks > lo) & (breaks < hi)]])
            for a, b in zip(cuts[:-1], cuts[1:]):
                xq, wq = _gauss_on(a, b)
                for x, wx in zip(xq, wq):
                    zs = []
                    for u, v in ((0, 1), (1, 2), (2, 0)):     # the facet's edges met by the line at x
                        xa, xb = P[u, 0], P[v, 0]
                        if xa != xb and min(xa, xb) <= x <= max(xa, xb):
                            zs.append(P[u, 1] + (x - xa) / (xb - xa) * (P[v, 1] - P[u, 1]))
                    zq, wz = _gauss_on(min(zs), max(zs))
                    pts = np.c_[np.full_like(zq, x), zq]
                    l12 = np.linalg.solve(T, (pts - P[0]).T).T
                    lam = np.c_[1.0 - l12.sum(1), l12]
                    _accumulate(f, lam, wx * wz, pts[:, 0], pp, pn, p, gp, gn)


def _accumulate(f, lam, w, x, pp, pn, p: Params, gp, gn):
    """gp[f[i]] += sum_q w_q p_p(x_q) (g_p + 2 h_p phi_p(x_q)) lam[q, i], and the same for NFA."""
    pref_p, pref_n = substrate_preference(x, p.Lx)
    php, phn = lam @ pp[f], lam @ pn[f]
    vp = w * pref_p * (p.g_p + 2.0 * p.h_p * php)
    vn = w * pref_n * (p.g_nfa + 2.0 * p.h_nfa * phn)
    np.add.at(gp, f, vp @ lam)
    np.add.at(gn, f, vn @ lam)


def boundary_load(m: Mesh, pp: np.ndarray, pn: np.ndarray, p: Params):
    """g_s[i] = int_{Gamma_b} (g_s + 2 h_s phi_s) lambda_i + evap_sign k int_{Gamma_t} phi_s phi_solv lambda_i.

    Flux boundary conditions of Eq. (10) with the substrate density of Eq. (5)
    (p(x) = 1, or Section 4's pattern when ``p.pattern``) and the evaporation flux
    k phi_i phi_s; readings R5, R6.
    Returns zeros when bc_mode == 0.
    """
    N = m.coords.shape[0]
    gp, gn = np.zeros(N), np.zeros(N)
    if p.bc_mode == 0:
        return gp, gn
    dF = m.dim - 1
    T1, T2, T3 = monomial_table(dF, 1), monomial_table(dF, 2), monomial_table(dF, 3)
    # substrate, Gamma_b
    if p.pattern:
        _patterned_substrate(m, pp, pn, p, gp, gn)
    else:
        Fb = m.bottom
        ab = facet_measure(m.coords[Fb])
        for g_s, h_s, phi, out in ((p.g_p, p.h_p, pp, gp), (p.g_nfa, p.h_nfa, pn, gn)):
            val = g_s * T1[None, :] + 2.0 * h_s * np.einsum("fa,ai->fi", phi[Fb], T2)
            np.add.at(out, Fb, ab[:, None] * val)
    # evaporation, Gamma_t
    Ft = m.top
    at = facet_measure(m.coords[Ft])
    solv = (1.0 - pp - pn)[Ft]
    for phi, out in ((pp, gp), (pn, gn)):
        val = p.evap_sign * p.k_evap * np.einsum("fa,fb,abi->fi", phi[Ft], solv, T3)
        np.add.at(out, Ft, at[:, None] * val)
    return gp, gn


# ----------------------------------------------------------------------------
# The saddle-point system of one species, Eq. (14)
# ----------------------------------------------------------------------------
def coefficients(p: Params):
    """(a, c) with A = [[M, a K], [a K, -c M]]: a = tau*mob, c = tau*mob/eps (Eq. (14))."""
    a = p.tau * p.mobility
    return a, a / p.eps


def saddle_matrix(M, K, p: Params):
    a, c = coefficients(p)
    return sp.bmat([[M, a * K], [a * K, -c * M]], format="csr")


def rhs(M, phi_k, F, gbd, p: Params):
    """b = [M phi^k + tau g_bd ; -(tau mob/eps) F^k] (Eq. (13) -> Eq. (14))."""
    _, c = coefficients(p)
    return np.concatenate([M @ phi_k + p.tau * gbd, -c * F])


def schur(M, K, p: Params):
    """Dense S = c M + a^2 K M^{-1} K, the Schur complement of A (Section 3)."""
    a, c = coefficients(p)
    Md, Kd = M.toarray(), K.toarray()
    return c * Md + a * a * Kd @ np.linalg.solve(Md, Kd)


def schur_tilde(M, K, p: Params):
    """Dense S~ = (a K + sqrt(c) M) M^{-1} (a K + sqrt(c) M), the matching approximation."""
    a, c = coefficients(p)
    Md = M.toarray()
    Hd = a * K.toarray() + math.sqrt(c) * Md
    return Hd @ np.linalg.solve(Md, Hd)


def mass(M, phi):
    """int_Omega phi_h = 1^T M phi."""
    return float(np.ones(M.shape[0]) @ (M @ phi))


# ----------------------------------------------------------------------------
# Time stepping (Eq. (12)/(13)), exact solve per step
# ----------------------------------------------------------------------------
@dataclass
class State:
    phi_p: np.ndarray
    phi_nfa: np.ndarray
    mu_p: np.ndarray
    mu_nfa: np.ndarray

    @property
    def phi_s(self):
        return 1.0 - self.phi_p - self.phi_nfa   # Eq. (2)


class Solver:
    """Mesh, matrices and a factorisation of A, reused across steps (A is constant)."""

    def __init__(self, p: Params, m: Mesh | None = None, factor: bool = True):
        self.p = p
        self.m = m if m is not None else mesh(p)
        self.M, self.K = assemble(self.m)
        self.A = saddle_matrix(self.M, self.K, p)
        self.N = self.M.shape[0]
        self._dense = self._lu = None
        if not factor:          # residual checks only (relres, rhs_pair); step() unavailable
            return
        if 2 * self.N <= DENSE_LIMIT:
            self._dense = self.A.toarray()
            self._lu = None
        else:
            self._dense = None
            self._lu = spla.splu(self.A.tocsc())

    def solve(self, B: np.ndarray) -> np.ndarray:
        if self._dense is None and self._lu is None:
            raise RuntimeError("Solver built with factor=False")
        if self._dense is not None:
            return np.linalg.solve(self._dense, B)     # LAPACK LU with partial pivoting
        return self._lu.solve(B)

    def rhs_pair(self, s: State):
        if self.p.potential == "fh":     # the logarithmic potential of Section 2 (reading R14)
            Fp, Fn = load_vector_fh(self.m, s.phi_p, s.phi_nfa, self.p)
        else:
            Fp, Fn = load_vector(self.m, s.phi_p, s.phi_nfa, self.p.potential)
        gp, gn = boundary_load(self.m, s.phi_p, s.phi_nfa, self.p)
        return (rhs(self.M, s.phi_p, Fp, gp, self.p), rhs(self.M, s.phi_nfa, Fn, gn, self.p))

    def step(self, s: State) -> State:
        bp, bn = self.rhs_pair(s)
        X = self.solve(np.stack([bp, bn], 1))
        N = self.N
        return State(X[:N, 0].copy(), X[:N, 1].copy(), X[N:, 0].copy(), X[N:, 1].copy())

    def run(self, s: State, nsteps: int):
        out = [s]
        for _ in range(nsteps):
            s = self.step(s)
            out.append(s)
        return out

    def relres(self, s_old: State, s_new: State):
        """True relative residuals ||b - A x|| / ||b|| of a candidate step solution, per species."""
        bp, bn = self.rhs_pair(s_old)
        out = []
        for b, phi, mu in ((bp, s_new.phi_p, s_new.mu_p), (bn, s_new.phi_nfa, s_new.mu_nfa)):
            r = b - self.A @ np.concatenate([phi, mu])
            out.append(float(np.linalg.norm(r) / np.linalg.norm(b)))
        return out


def initial(n_nodes: int, phi_p: np.ndarray, phi_nfa: np.ndarray) -> State:
    """Initial state from given nodal fractions; mu^0 = 0 (mu^0 never enters b)."""
    return State(np.asarray(phi_p, float).copy(), np.asarray(phi_nfa, float).copy(),
                 np.zeros(n_nodes), np.zeros(n_nodes))


# ----------------------------------------------------------------------------
# Algorithm 1 with exact inner solves (the ideal form of the preconditioner)
# ----------------------------------------------------------------------------
def algorithm1_exact(M, K, p: Params, v1: np.ndarray, v2: np.ndarray):
    """Prec(v) of Algorithm 1 with every "approximately solve" replaced by an exact solve:
    w1 = M^-1 v1;  w2 = H^-1 v2;  w2 <- M w2;  w2 = H^-1 w2, with H = a K + sqrt(c) M.
    v1, v2 may be (N,) or (N, r)."""
    a, c = coefficients(p)
    H = (a * K + math.sqrt(c) * M).tocsc()
    w1 = spla.spsolve(M.tocsc(), v1)
    w2 = spla.spsolve(H, v2)
    w2 = M @ w2
    w2 = spla.spsolve(H, w2)
    return w1, w2


# ----------------------------------------------------------------------------
# M~ by a Chebyshev semi-iteration (Section 3: the alternative to AMG for the
# mass matrix; Wathen & Rees 2008)
# ----------------------------------------------------------------------------
WATHEN_BOUNDS = {2: (0.5, 2.0), 3: (0.5, 2.5)}  # eig(D^-1 M) for P1 triangles / tetrahedra


def chebyshev_semi_iteration(M, b: np.ndarray, steps: int, bounds=None, dim: int = 2):
    """x_k ~ M^-1 b by k steps of the Chebyshev semi-iteration on the Jacobi-preconditioned system
    D^-1 M x = D^-1 b (D = diag(M)), started from x_0 = 0, for eigenvalues of D^-1 M in
    [lo, hi] (default: Wathen's bounds for the element type).

    The iterate is x_k = q_k(D^-1 M) D^-1 b with 1 - t q_k(t) = T_k((th - t) / de) / T_k(th / de),
    th = (hi + lo) / 2, de = (hi - lo) / 2: the residual polynomial of least maximum on
    [lo, hi].  It is computed by the three-term recurrence of the Chebyshev polynomials
    (x_{k+1} = x_k + d_k with d_k mixing d_{k-1} and the preconditioned residual)."""
    lo, hi = bounds if bounds is not None else WATHEN_BOUNDS[dim]
    th, de = 0.5 * (hi + lo), 0.5 * (hi - lo)
    sigma = th / de
    dinv = 1.0 / M.diagonal()
    x = np.zeros_like(b, dtype=np.float64)
    if steps <= 0:
        return x
    dinv_b = dinv[:, None] * b if b.ndim == 2 else dinv * b
    d = dinv_b / th                       # first step: Jacobi damped by 1 / th
    rho = 1.0 / sigma
    x = x + d
    for _ in range(1, steps):
        r = b - M @ x
        z = dinv[:, None] * r if r.ndim == 2 else dinv * r
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / de) * z
        x = x + d
        rho = rho_new
    return x


# ----------------------------------------------------------------------------
# The Flory-Huggins bulk energy (the logarithmic potential of Section 2, which the
# paper's experiments replace by Eq. (15)) and its load by a fixed quadrature rule
# ----------------------------------------------------------------------------
def _guarded_log(x, delta):
    return np.log(np.maximum(x, delta))


def flory_huggins(pp: np.ndarray, pn: np.ndarray, p: Params):
    """f(phi_p, phi_nfa, phi_s) with phi_s = 1 - phi_p - phi_nfa: the entropic terms phi ln(phi) / N
    and the pairwise interactions chi phi phi'; logarithms guarded at fh_delta."""
    ps = 1.0 - pp - pn
    dl = p.fh_delta
    return (pp / p.N_p * _guarded_log(pp, dl) + pn / p.N_nfa * _guarded_log(pn, dl)
            + ps / p.N_s * _guarded_log(ps, dl)
            + p.chi_pn * pp * pn + p.chi_ps * pp * ps + p.chi_ns * pn * ps)


def dfdphi_fh(pp: np.ndarray, pn: np.ndarray, p: Params):
    """df/dphi_p and df/dphi_nfa of the Flory-Huggins f through phi_s = 1 - phi_p - phi_nfa
    (the chain rule of reading R3):
      f_p' = (ln phi_p + 1)/N_p - (ln phi_s + 1)/N_s + chi_pn phi_n + chi_ps (phi_s - phi_p) - chi_ns phi_n
      f_n' = (ln phi_n + 1)/N_n - (ln phi_s + 1)/N_s + chi_pn phi_p - chi_ps phi_p + chi_ns (phi_s - phi_n)."""
    ps = 1.0 - pp - pn
    dl = p.fh_delta
    ls = (_guarded_log(ps, dl) + 1.0) / p.N_s
    fp = ((_guarded_log(pp, dl) + 1.0) / p.N_p - ls + p.chi_pn * pn + p.chi_ps * (ps - pp) - p.chi_ns * pn)
    fn = ((_guarded_log(pn, dl) + 1.0) / p.N_nfa - ls + p.chi_pn * pp - p.chi_ps * pp + p.chi_ns * (ps - pn))
    return fp, fn


def simplex_gauss_rule(d: int, n: int = 3):
    """Collapsed (Duffy) Gauss-Legendre product rule on a d-simplex with n points per direction:
    barycentric points (n^d, d+1) and weights summing to 1, so int_T g = |T| sum_q w_q g(x_q).
    Exact for polynomials of degree 2n - d (the collapse adds d - 1 to the degree in the first
    direction): 4 in 2D, 3 in 3D for n = 3."""
    g, w = np.polynomial.legendre.leggauss(n)
    g, w = 0.5 * (g + 1.0), 0.5 * w
    if d == 2:
        u, v = np.meshgrid(g, g, indexing="ij")
        wu, wv = np.meshgrid(w, w, indexing="ij")
        xi = np.c_[u.ravel(), (v * (1 - u)).ravel()]
        wt = 2.0 * (wu * wv * (1 - u)).ravel()
    elif d == 3:
        u, v, t = np.meshgrid(g, g, g, indexing="ij")
        wu, wv, wt3 = np.meshgrid(w, w, w, indexing="ij")
        xi = np.c_[u.ravel(), (v * (1 - u)).ravel(), (t * (1 - u) * (1 - v)).ravel()]
        wt = 6.0 * (wu * wv * wt3 * (1 - u) ** 2 * (1 - v)).ravel()
    else:
        raise ValueError("d must be 2 or 3")
    return np.c_[1.0 - xi.sum(1), xi], wt


def load_vector_fh(m: Mesh, pp: np.ndarray, pn: np.ndarray, p: Params, n: int = 3):
    """F_s[i] = int df/dphi_s(phi_h) lambda_i for the Flory-Huggins f, each simplex integrated by
    simplex_gauss_rule(d, n) (the rule defines the load: the integrand is not a polynomial)."""
    d = m.dim
    N = m.coords.shape[0]
    vol, _ = simplex_measure_and_gradients(m.coords[m.elems])
    lam, w = simplex_gauss_rule(d, n)                           # (Q, d+1), (Q,)
    php = pp[m.elems] @ lam.T                                   # (E, Q) phi_h at the points
    phn = pn[m.elems] @ lam.T
    fp, fn = dfdphi_fh(php, phn, p)
    Fp, Fn = np.zeros(N), np.zeros(N)
    np.add.at(Fp, m.elems, vol[:, None] * ((fp * w) @ lam))
    np.add.at(Fn, m.elems, vol[:, None] * ((fn * w) @ lam))
    return Fp, Fn


# ----------------------------------------------------------------------------
# A multigrid V-cycle over a given hierarchy (the inner solves of Algorithm 1)
# ----------------------------------------------------------------------------
def chebyshev_smooth(A, b: np.ndarray, x0: np.ndarray, degree: int, bounds):
    """`degree` Chebyshev steps on D^-1 A x = D^-1 b from x0 for eigenvalues of D^-1 A in
    [lo, hi]: x = x0 + q(D^-1 A) D^-1 (b - A x0), q the semi-iteration's polynomial."""
    return x0 + chebyshev_semi_iteration(A, b - A @ x0, degree, bounds=bounds)


def vcycle(levels, b: np.ndarray, x0: np.ndarray | None = None, level: int = 0):
    """One V-cycle for A_0 x = b.  levels[l] = dict(A=A_l, P=P_l (rows of level l x rows of
    level l+1), bounds=(lo, hi), degree=k) for every level but the last, whose dict holds only A
    (solved exactly).  Per level: pre-smooth, restrict the residual with P^T, recurse from zero,
    prolongate the correction, post-smooth with the same polynomial."""
    L = levels[level]
    A = L["A"]
    if level == len(levels) - 1:
        return np.linalg.solve(A.toarray() if sp.issparse(A) else A, b)
    x = np.zeros_like(b, dtype=np.float64) if x0 is None else x0
    x = chebyshev_smooth(A, b, x, L["degree"], L["bounds"])
    r_c = L["P"].T @ (b - A @ x)
    e_c = vcycle(levels, r_c, None, level + 1)
    x = x + L["P"] @ e_c
    return chebyshev_smooth(A, b, x, L["degree"], L["bounds"])


def galerkin_levels(A, Ps, bounds_list, degrees):
    """levels for `vcycle` from the fine matrix and prolongators: A_{l+1} = P_l^T A_l P_l."""
    levels = []
    for P, bd, k in zip(Ps, bounds_list, degrees):
        levels.append(dict(A=A, P=P, bounds=bd, degree=k))
        A = (P.T @ A @ P).tocsr()
    levels.append(dict(A=A))
    return levels
