"""Structured-grid FIT stand-in for the paper's hp-FEM discretisation.

The paper discretises the regularised transmission problem (Sect. 3, Eq. (7))
with H(curl)-conforming hp finite elements and obtains the real symmetric
sparse matrices K (curl-curl stiffness, Eq. (10a)), C (conductivity "damping"
matrix on the object B, Eq. (10b)) and M (regularisation mass on the exterior,
Eq. (10c)).  Meshes and NGSolve are not available here, so this module builds
the lowest-order edge (finite integration) analogue on an n^3 grid of the unit
box Omega = [-1/2, 1/2]^3 (dimensionless coordinates xi, origin at the box
centre, which lies inside B):

* DOFs are tangential components on interior edges; edges on the outer
  boundary are eliminated (n x theta = 0 on dOmega, Eq. (7d)), so
  N = 3 n (n-1)^2.
* K = G^T diag(h * mean(mu_r^-1 of the two cells)) G, where G is the signed
  face-edge incidence (discrete curl).  This is the lowest-order curl-curl form
  with lumped face mass: real, symmetric, positive semi-definite.
* C = diag(alpha^2 mu_0 sum_{cells c touching e} sigma_c h^3 / 4)   (lumped).
* M = diag(sum_{cells c touching e, sigma_c = 0} h^3 / 4)            (lumped).
* x_i = edge values of e_i x xi (exact for lowest-order edge elements, since
  the field is linear), and, for mu_r != 1, the static correction
  o~_i solving (K + eps_s M_Omega) o~_i = -K x_i, so that the total
  theta^(0) coefficients are o_i = x_i + o~_i (Sect. 3, below Eq. (5)).
* N0 follows Eq. (6a) with the same lumped quadrature.
* Optionally (mu_split=True) the part K_in of K carried by the cells of the
  object B (the conducting cells), so that scaling mu_r on B by s gives
  K(s) = (K - K_in) + K_in / s, with the matching parts of K x (boundary
  columns included) for the static right-hand side; mu_scale and
  sigma_scale build the problem at scaled material parameters.

This is problem data (the discretised PDE), not the reduced-order method.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Sequence

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

MU0 = 4.0e-7 * np.pi


@dataclass(frozen=True)
class Material:
    """Axis-aligned box of material in box coordinates [0,1]^3 (cell centres inside are assigned)."""

    lo: tuple
    hi: tuple
    sigma: float
    mu_r: float


# Centred cube [0.375, 0.625]^3, sigma = 5.96e7 S/m, mu_r = 1 (the 16^3 FP64 case).
CUBE_C1 = (Material((0.375,) * 3, (0.625,) * 3, 5.96e7, 1.0),)
# Centred cube [0.375, 0.625]^3, sigma = 1.5e6 S/m, mu_r = 32 (the 96^3 precision case).
CUBE_C2 = (Material((0.375,) * 3, (0.625,) * 3, 1.5e6, 32.0),)
# Shell [0.375,0.625]^3 minus inner cube, sigma 3.5e7, mu_r 1; inner cube
# [0.4375,0.5625]^3, sigma 1e6, mu_r 64 (later entries override earlier ones).
TWO_MATERIAL_C5 = (
    Material((0.375,) * 3, (0.625,) * 3, 3.5e7, 1.0),
    Material((0.4375,) * 3, (0.5625,) * 3, 1.0e6, 64.0),
)


@dataclass
class FitProblem:
    """Discretised eddy-current problem on an n^3 FIT grid (all arrays float64)."""

    n: int
    h: float
    alpha: float
    eps: float
    K: sp.csr_matrix            # N x N curl-curl stiffness (interior edges)
    C: np.ndarray               # N, lumped conductivity mass (diagonal of C)
    M: np.ndarray               # N, lumped exterior mass (diagonal of M)
    M_omega: np.ndarray         # N, lumped mass over all of Omega
    x: np.ndarray               # 3 x N, edge values of e_i x xi
    o_tilde: np.ndarray         # 3 x N, static correction (0 when mu_r == 1)
    N0: np.ndarray              # 3 x 3, Eq. (6a)
    cell_sigma: np.ndarray      # n^3
    cell_mu: np.ndarray         # n^3
    edge_dir: np.ndarray        # N, 0/1/2 = x/y/z edge
    edge_mid: np.ndarray        # N x 3, edge mid-points in xi coordinates
    vol_B: float                # |B| (dimensionless volume of conducting cells)
    extra: dict = field(default_factory=dict)
    eps_static: float = 1e-10   # regularisation of the static theta^(0) problem (mass on Omega)
    K_in: sp.csr_matrix | None = None   # N x N part of K carried by the cells of B (mu_split)
    kx: np.ndarray | None = None        # 3 x N, rows of K x with the boundary columns (mu_split)
    kx_in: np.ndarray | None = None     # 3 x N, the part of kx carried by the cells of B (mu_split)
    vol_B_mu: float = 0.0               # sum over the cells of B of |cell| / mu_r (mu_split)

    @property
    def N(self) -> int:
        return self.K.shape[0]

    @property
    def o(self) -> np.ndarray:
        """Total theta^(0) coefficients o_i = x_i + o~_i (3 x N)."""
        return self.x + self.o_tilde

    def A(self, omega: float) -> sp.csc_matrix:
        """A[omega] = K - i omega C + eps M (Sect. 3.1, below Eq. (9))."""
        return (self.K.astype(np.complex128)
                + sp.diags(self.eps * self.M - 1j * omega * self.C)).tocsc()

    def rhs(self, omega: float) -> np.ndarray:
        """Source r_i = i omega C o_i for the three directions (N x 3)."""
        return (1j * omega) * (self.C[:, None] * self.o.T)


def _edge_tables(n: int):
    """Enumerate all edges (boundary included) of the n^3 grid.

    Returns per-direction index arrays so that a node-lattice position maps to
    a global edge id: x-edges (i in [0,n), j,k in [0,n]), then y-edges, then
    z-edges.
    """
    shapes = [(n, n + 1, n + 1), (n + 1, n, n + 1), (n + 1, n + 1, n)]
    ids, off = [], 0
    for s in shapes:
        cnt = s[0] * s[1] * s[2]
        ids.append(np.arange(off, off + cnt).reshape(s))
        off += cnt
    return ids, off


def _curl_incidence(n: int, ids):
    """Signed face-edge incidence G (faces x all edges) and each face's two cells."""
    ex, ey, ez = ids
    rows, cols, vals = [], [], []
    cellA, cellB = [], []
    nf = 0

    def add(face_edges, signs, cA, cB):
        nonlocal nf
        m = face_edges[0].size
        fid = np.arange(nf, nf + m)
        for e, s in zip(face_edges, signs):
            rows.append(fid)
            cols.append(e.ravel())
            vals.append(np.full(m, s, dtype=np.float64))
        cellA.append(cA.ravel())
        cellB.append(cB.ravel())
        nf += m

    def cell(i, j, k):
        # cell id, or -1 outside the grid
        ok = (i >= 0) & (i < n) & (j >= 0) & (j < n) & (k >= 0) & (k < n)
        return np.where(ok, (i * n + j) * n + k, -1)

    # x-faces at node plane i, spanning (j,j+1) x (k,k+1): y -> z circulation
    I, J, Kk = np.meshgrid(np.arange(n + 1), np.arange(n), np.arange(n), indexing="ij")
    add([ey[I, J, Kk], ez[I, J + 1, Kk], ey[I, J, Kk + 1], ez[I, J, Kk]], [1, 1, -1, -1],
        cell(I - 1, J, Kk), cell(I, J, Kk))
    # y-faces at node plane j: z -> x circulation
    I, J, Kk = np.meshgrid(np.arange(n), np.arange(n + 1), np.arange(n), indexing="ij")
    add([ez[I, J, Kk], ex[I, J, Kk + 1], ez[I + 1, J, Kk], ex[I, J, Kk]], [1, 1, -1, -1],
        cell(I, J - 1, Kk), cell(I, J, Kk))
    # z-faces at node plane k: x -> y circulation
    I, J, Kk = np.meshgrid(np.arange(n), np.arange(n), np.arange(n + 1), indexing="ij")
    add([ex[I, J, Kk], ey[I + 1, J, Kk], ex[I, J + 1, Kk], ey[I, J, Kk]], [1, 1, -1, -1],
        cell(I, J, Kk - 1), cell(I, J, Kk))

    G = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(nf, sum(e.size for e in ids)))
    return G, np.concatenate(cellA), np.concatenate(cellB)


def _edge_cells(n: int, ids):
    """For every edge, the (up to four) cells that touch it (-1 where outside)."""
    ex, ey, ez = ids
    total = sum(e.size for e in ids)
    out = np.full((total, 4), -1, dtype=np.int64)
    mids = np.zeros((total, 3))
    dirs = np.zeros(total, dtype=np.int8)

    def cid(i, j, k):
        ok = (i >= 0) & (i < n) & (j >= 0) & (j < n) & (k >= 0) & (k < n)
        return np.where(ok, (i * n + j) * n + k, -1)

    h = 1.0 / n
    # x-edge (i,j,k): from node (i,j,k) to (i+1,j,k); cells (i, j-1..j, k-1..k)
    I, J, K = np.meshgrid(np.arange(n), np.arange(n + 1), np.arange(n + 1), indexing="ij")
    e = ex[I, J, K].ravel()
    out[e] = np.stack([cid(I, J - a, K - b).ravel() for a in (0, 1) for b in (0, 1)], 1)
    mids[e] = np.stack([((I + 0.5) * h).ravel(), (J * h).ravel(), (K * h).ravel()], 1)
    dirs[e] = 0
    I, J, K = np.meshgrid(np.arange(n + 1), np.arange(n), np.arange(n + 1), indexing="ij")
    e = ey[I, J, K].ravel()
    out[e] = np.stack([cid(I - a, J, K - b).ravel() for a in (0, 1) for b in (0, 1)], 1)
    mids[e] = np.stack([(I * h).ravel(), ((J + 0.5) * h).ravel(), (K * h).ravel()], 1)
    dirs[e] = 1
    I, J, K = np.meshgrid(np.arange(n + 1), np.arange(n + 1), np.arange(n), indexing="ij")
    e = ez[I, J, K].ravel()
    out[e] = np.stack([cid(I - a, J - b, K).ravel() for a in (0, 1) for b in (0, 1)], 1)
    mids[e] = np.stack([(I * h).ravel(), (J * h).ravel(), ((K + 0.5) * h).ravel()], 1)
    dirs[e] = 2
    return out, mids - 0.5, dirs


def node_gradient(n: int) -> sp.csr_matrix:
    """Discrete gradient of the n^3 grid restricted to interior edges and interior nodes
    (rows in the edge order of fit_problem, columns = interior nodes in lexicographic order):
    each edge holds phi(end) - phi(start) along its positive direction.  Boundary nodes carry
    phi = 0 (n x grad phi = 0 on the boundary), so K G = 0 for the curl-curl K of fit_problem."""
    ids, n_all = _edge_tables(n)
    ex, ey, ez = ids
    node = lambda i, j, k: (i * (n + 1) + j) * (n + 1) + k
    rows, cols, vals = [], [], []
    for d, e in enumerate(ids):
        I, J, K = np.meshgrid(*[np.arange(s) for s in e.shape], indexing="ij")
        start = node(I, J, K).ravel()
        step = [(1, 0, 0), (0, 1, 0), (0, 0, 1)][d]
        end = node(I + step[0], J + step[1], K + step[2]).ravel()
        eid = e[I, J, K].ravel()
        rows += [eid, eid]
        cols += [end, start]
        vals += [np.ones(eid.size), -np.ones(eid.size)]
    G = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n_all, (n + 1) ** 3))
    # interior edges: the same selection as fit_problem (mid-point off the outer faces)
    _, mids, dirs = _edge_cells(n, ids)
    on_bnd = np.zeros(n_all, dtype=bool)
    for d in range(3):
        sel = dirs == d
        for t in range(3):
            if t == d:
                continue
            coord = mids[sel, t] + 0.5
            on_bnd[np.flatnonzero(sel)[(np.abs(coord) < 1e-12) | (np.abs(coord - 1.0) < 1e-12)]] = True
    interior = np.flatnonzero(~on_bnd)
    a = np.arange(1, n)
    I, J, K = np.meshgrid(a, a, a, indexing="ij")
    inodes = node(I, J, K).ravel()
    return G[interior][:, inodes].tocsr()


def _assign_materials(n: int, materials: Sequence[Material]):
    h = 1.0 / n
    c = (np.arange(n) + 0.5) * h
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    sigma = np.zeros(n ** 3)
    mu = np.ones(n ** 3)
    for m in materials:
        inside = ((X >= m.lo[0]) & (X < m.hi[0]) & (Y >= m.lo[1]) & (Y < m.hi[1])
                  & (Z >= m.lo[2]) & (Z < m.hi[2])).ravel()
        sigma[inside] = m.sigma
        mu[inside] = m.mu_r
    return sigma, mu


def fit_problem(n: int, materials: Sequence[Material] = CUBE_C1, *, alpha: float = 1.0,
                eps: float = 1e-6, eps_static: float = 1e-10,
                static_solver: Callable | None = None, static: bool = True,
                mu_scale: float = 1.0, sigma_scale: float = 1.0, mu_split: bool = False) -> FitProblem:
    """Assemble the FIT problem on an n^3 grid.

    eps is the regularisation of Eq. (7b) (mass on Omega minus B); eps_static
    regularises the static theta^(0) problem with mass on all of Omega (M_s = eps_static M_Omega);
    static_solver(K, M_s, rhs) -> o~ (N x 3) replaces the default sparse LU for that problem, whose
    solution is the one with G^T M_s o~ = 0 for the discrete gradient G.  The
    static solve is skipped (o~ = 0, N0 = 0) when mu_r == 1 everywhere, or when
    static=False (for grids too large for a sparse direct solve; the operator
    shapes are unchanged).  mu_scale multiplies mu_r and sigma_scale sigma in
    every conducting cell; mu_split adds K_in, kx, kx_in and vol_B_mu.
    """
    if n < 2:
        raise ValueError("n must be >= 2")
    h = 1.0 / n
    ids, n_all = _edge_tables(n)
    G, cA, cB = _curl_incidence(n, ids)
    ecells, mids, dirs = _edge_cells(n, ids)
    sigma, mu = _assign_materials(n, materials)
    in_B = sigma > 0.0
    sigma = sigma * sigma_scale
    mu = np.where(in_B, mu * mu_scale, mu)

    # interior edges: mid-point strictly inside in the two transverse coordinates
    on_bnd = np.zeros(n_all, dtype=bool)
    for d in range(3):
        sel = dirs == d
        for t in range(3):
            if t == d:
                continue
            coord = mids[sel, t] + 0.5
            on_bnd[np.flatnonzero(sel)[(np.abs(coord) < 1e-12) | (np.abs(coord - 1.0) < 1e-12)]] = True
    interior = np.flatnonzero(~on_bnd)

    inv_mu = 1.0 / mu
    wA = np.where(cA >= 0, inv_mu[np.maximum(cA, 0)], np.nan)
    wB = np.where(cB >= 0, inv_mu[np.maximum(cB, 0)], np.nan)
    face_w = h * np.nanmean(np.stack([wA, wB]), axis=0)
    Kall = (G.T @ sp.diags(face_w) @ G).tocsr()
    K = Kall[interior][:, interior].tocsr()
    K.sum_duplicates()
    K.eliminate_zeros()

    v4 = h ** 3 / 4.0
    ok = ecells >= 0
    sig_e = np.where(ok, sigma[np.maximum(ecells, 0)], 0.0)
    C_all = alpha ** 2 * MU0 * v4 * sig_e.sum(1)
    M_all = v4 * (ok & (sig_e == 0.0)).sum(1)
    Mo_all = v4 * ok.sum(1)

    xi = mids
    x_all = np.zeros((3, n_all))
    # tangential component of e_i x xi along each edge direction
    ecross = lambda i, p: np.cross(np.eye(3)[i], p)
    for i in range(3):
        v = ecross(i, xi)
        x_all[i] = v[np.arange(n_all), dirs]

    N = interior.size
    split = {}
    if mu_split:
        # each face weight is the mean of its cells' mu_r^-1; the share of the cells of B
        cnt = (cA >= 0).astype(np.float64) + (cB >= 0)
        wA_in = np.where((cA >= 0) & in_B[np.maximum(cA, 0)], inv_mu[np.maximum(cA, 0)], 0.0)
        wB_in = np.where((cB >= 0) & in_B[np.maximum(cB, 0)], inv_mu[np.maximum(cB, 0)], 0.0)
        Kin_all = (G.T @ sp.diags(h * (wA_in + wB_in) / cnt) @ G).tocsr()
        K_in = Kin_all[interior][:, interior].tocsr()
        K_in.sum_duplicates()
        split = dict(K_in=K_in, kx=np.asarray(Kall[interior] @ x_all.T).T.copy(),
                     kx_in=np.asarray(Kin_all[interior] @ x_all.T).T.copy(),
                     vol_B_mu=float(np.sum(inv_mu[in_B]) * h ** 3))
    o_tilde = np.zeros((3, N))
    N0 = np.zeros((3, 3))
    magnetic = np.any(mu != 1.0)
    if magnetic and static:
        Kia = Kall[interior]
        rhs = -(Kia @ x_all.T)
        Ms = eps_static * Mo_all[interior]
        if static_solver is not None:
            o_tilde = np.asarray(static_solver(K, Ms, rhs)).T
        else:
            # sparse LU of K + M_s, then the gradient part fixed exactly: K G = 0 leaves it to the
            # tiny M_s, so the LU solution carries rounding there of about cond x eps; the solution
            # satisfies G^T M_s o~ = 0, restored by o~ -= G (G^T M_s G)^-1 G^T M_s o~
            o_t = spla.splu((K + sp.diags(Ms)).tocsc()).solve(rhs)
            Gn = node_gradient(n)
            Ln = (Gn.T @ sp.diags(Ms) @ Gn).tocsc()
            o_t = o_t - Gn @ spla.splu(Ln).solve(np.asarray(Gn.T @ (Ms[:, None] * o_t)))
            o_tilde = np.asarray(o_t).T
        N0 = alpha ** 3 * np.eye(3) * np.sum(1.0 - inv_mu) * h ** 3 \
            + alpha ** 3 / 4.0 * (o_tilde @ (K @ o_tilde.T))

    return FitProblem(
        n=n, h=h, alpha=alpha, eps=eps, K=K, C=C_all[interior], M=M_all[interior],
        M_omega=Mo_all[interior], x=x_all[:, interior], o_tilde=o_tilde, N0=N0,
        cell_sigma=sigma, cell_mu=mu, edge_dir=dirs[interior], edge_mid=mids[interior],
        vol_B=float(np.count_nonzero(sigma > 0) * h ** 3), eps_static=eps_static, **split,
    )
