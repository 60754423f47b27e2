"""Finite-element matrices of the diffusion sub-problem (Eq. 2b, 2c).

The stiffness matrix K has entries k_ij = sum_e int_e grad(N_i) . D_e grad(N_j)
and the mass matrix m_ij = sum_e int_e N_i N_j.  Section 2 uses the diagonal
entries m_ii in Eq. 3 and advances V with explicit Euler, which needs a
diagonal mass; the oracle therefore uses the row-sum lumped mass
m_i = sum_j m_ij (the paper does not name the lumping; this reading reproduces
the dt_s = 0.013 ms printed in Section 3.1).

Elements: 4-node bilinear quads (Section 3.1, 3.2), 8-node trilinear hexes
(structured 3D slab) and 4-node linear tetrahedra (Section 3.3), all with an
element-constant tensor D_e = d_t I + (d_l - d_t) f f^T (fibre f, longitudinal
d_l, transverse d_t = rho d_l; Section 3.1).
"""
from __future__ import annotations

import itertools

import numpy as np
import scipy.sparse as sp

_G = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])   # 2-point Gauss on [0, 1]
_W = np.array([0.5, 0.5])


def conductivity_tensor(d_long, d_trans, fibre, dim):
    """D = d_t I + (d_l - d_t) f f^T for each element; returns (n_elem, dim, dim)."""
    d_long = np.asarray(d_long, dtype=np.float64)
    d_trans = np.asarray(d_trans, dtype=np.float64)
    f = np.asarray(fibre, dtype=np.float64)[:, :dim]
    nrm = np.linalg.norm(f, axis=1, keepdims=True)
    f = np.where(nrm > 0, f / np.where(nrm > 0, nrm, 1.0), 0.0)
    eye = np.eye(dim)[None, :, :]
    return d_trans[:, None, None] * eye + (d_long - d_trans)[:, None, None] * (f[:, :, None] * f[:, None, :])


def _tensor_shape(dim):
    """Local node a of the reference cube has coordinates bits(a) = (a&1, a>>1&1, a>>2&1)."""
    return [tuple((a >> d) & 1 for d in range(dim)) for a in range(2 ** dim)]


def _shape_and_grad(dim, xi):
    """Values N_a(xi) and reference gradients dN_a/dxi on the unit square/cube."""
    corners = _tensor_shape(dim)
    N = np.empty(len(corners))
    dN = np.empty((len(corners), dim))
    for a, c in enumerate(corners):
        f1 = [xi[d] if c[d] else 1.0 - xi[d] for d in range(dim)]
        df = [1.0 if c[d] else -1.0 for d in range(dim)]
        N[a] = np.prod(f1)
        for d in range(dim):
            g = df[d]
            for e in range(dim):
                if e != d:
                    g *= f1[e]
            dN[a, d] = g
    return N, dN


def box_element_matrices(dim, h, D):
    """Stiffness (from tensor D) and consistent mass of an axis-aligned square/cube of side h.

    Tensor-product 2-point Gauss rule per axis: exact, the integrands are at most
    quadratic per coordinate.
    """
    nloc = 2 ** dim
    K = np.zeros((nloc, nloc))
    M = np.zeros((nloc, nloc))
    for q in itertools.product(range(2), repeat=dim):
        xi = [_G[i] for i in q]
        w = np.prod([_W[i] for i in q])
        N, dN = _shape_and_grad(dim, xi)
        grad = dN / h                                   # physical gradients
        K += w * h ** dim * grad @ D @ grad.T
        M += w * h ** dim * np.outer(N, N)
    return K, M


def tet_element_matrices(X, D):
    """P1 tetrahedron with vertices X (4 x 3): K = |e| G D G^T, M = |e|/20 (1 + delta_ab)."""
    J = (X[1:] - X[0]).T                                 # columns: edge vectors
    vol = abs(np.linalg.det(J)) / 6.0
    Jinv = np.linalg.inv(J)                              # rows: gradients of lambda_1..3
    G = np.vstack([-Jinv.sum(axis=0), Jinv])
    K = vol * G @ D @ G.T
    M = vol / 20.0 * (np.ones((4, 4)) + np.eye(4))
    return K, M


def grid_elements(dim, n):
    """Global node numbers of each box element in local order (bits of a = x, y, z offsets)."""
    nx, ny = n[0], n[1]
    nz = n[2] if dim == 3 else 1
    ez_n = (nz - 1) if dim == 3 else 1
    ez, ey, ex = np.meshgrid(np.arange(ez_n), np.arange(ny - 1), np.arange(nx - 1), indexing="ij")
    base = (ex + nx * (ey + ny * ez)).ravel()
    offs = []
    for c in _tensor_shape(dim):
        cz = c[2] if dim == 3 else 0
        offs.append(c[0] + nx * c[1] + nx * ny * cz)
    return base[:, None] + np.array(offs)[None, :]


def assemble(conn, Ke_list, Me_list, n_nodes):
    """Sum element matrices into global CSR K and consistent CSR M."""
    nloc = conn.shape[1]
    rows = np.repeat(conn, nloc, axis=1).ravel()
    cols = np.tile(conn, (1, nloc)).ravel()
    K = sp.csr_matrix((np.asarray(Ke_list).ravel(), (rows, cols)), shape=(n_nodes, n_nodes))
    M = sp.csr_matrix((np.asarray(Me_list).ravel(), (rows, cols)), shape=(n_nodes, n_nodes))
    K.sum_duplicates()
    M.sum_duplicates()
    return K, M


def assemble_grid(dim, n, h, d_long, d_trans, fibre):
    """K, lumped mass m for a structured grid with per-element conductivity."""
    conn = grid_elements(dim, n)
    Ds = conductivity_tensor(d_long, d_trans, fibre, dim)
    # group identical tensors to keep the element loop small
    keys, inv = np.unique(np.round(Ds.reshape(len(Ds), -1), 18), axis=0, return_inverse=True)
    inv = np.asarray(inv).ravel()
    Kref, Mref = [], None
    for kk in keys:
        Ke, Me = box_element_matrices(dim, h, kk.reshape(dim, dim))
        Kref.append(Ke)
        Mref = Me
    Ke_all = np.asarray(Kref)[inv]
    Me_all = np.broadcast_to(Mref, Ke_all.shape)
    n_nodes = int(np.prod(n[:dim]))
    K, M = assemble(conn, Ke_all, Me_all, n_nodes)
    m = np.asarray(M.sum(axis=1)).ravel()
    return K, m


def assemble_tets(xyz, tets, d_long, d_trans, fibre):
    """K, lumped mass m for a P1 tetrahedral mesh with per-element conductivity."""
    Ds = conductivity_tensor(d_long, d_trans, fibre, 3)
    Ke_all = np.empty((len(tets), 4, 4))
    Me_all = np.empty((len(tets), 4, 4))
    for e in range(len(tets)):
        Ke_all[e], Me_all[e] = tet_element_matrices(xyz[tets[e]], Ds[e])
    K, M = assemble(np.asarray(tets), Ke_all, Me_all, xyz.shape[0])
    m = np.asarray(M.sum(axis=1)).ravel()
    return K, m


def assemble_tets_vectorised(xyz, tets, d_long, d_trans, fibre):
    """Same as ``assemble_tets`` with the per-element algebra batched (large meshes)."""
    Ds = conductivity_tensor(d_long, d_trans, fibre, 3)
    X = xyz[tets]                                        # (ne, 4, 3)
    J = np.transpose(X[:, 1:, :] - X[:, :1, :], (0, 2, 1))
    vol = np.abs(np.linalg.det(J)) / 6.0
    Jinv = np.linalg.inv(J)
    G = np.concatenate([-Jinv.sum(axis=1, keepdims=True), Jinv], axis=1)   # (ne, 4, 3)
    Ke_all = vol[:, None, None] * np.einsum("eai,eij,ebj->eab", G, Ds, G)
    Me_all = (vol / 20.0)[:, None, None] * (np.ones((4, 4)) + np.eye(4))[None]
    K, M = assemble(np.asarray(tets), Ke_all, Me_all, xyz.shape[0])
    m = np.asarray(M.sum(axis=1)).ravel()
    return K, m


def assemble_workload(wl):
    """K, m for an ``inputs.Workload`` (structured grid or tet mesh)."""
    if wl.tets is not None:
        return assemble_tets_vectorised(wl.xyz, wl.tets, wl.d_long, wl.d_trans, wl.fibre)
    return assemble_grid(wl.dim, wl.n, wl.h, wl.d_long, wl.d_trans, wl.fibre)
