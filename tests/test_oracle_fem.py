"""Pins of the oracle's finite-element assembly (Section 2, Eq. 3; Section 3).

Each check is fixed by mathematics or by a number printed in the paper, not
by re-typing the oracle's own formulas.
"""
import json
import math
import os

import numpy as np
import pytest

import inputs as I
from oracle import fem, scheme

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_bilinear_isotropic_closed_form():
    # textbook bilinear-quad Laplacian: 2/3 on the diagonal, -1/6 to edge
    # neighbours, -1/3 to the diagonal neighbour; independent of h in 2D
    for h in (0.01, 0.3):
        K, M = fem.box_element_matrices(2, h, np.eye(2) * 2.0)
        exp = 2.0 * np.array([[4, -1, -1, -2], [-1, 4, -2, -1], [-1, -2, 4, -1], [-2, -1, -1, 4]]) / 6.0
        np.testing.assert_allclose(K, exp, atol=1e-14)
        np.testing.assert_allclose(M.sum(axis=1), np.full(4, h * h / 4), rtol=1e-14)
        # consistent bilinear mass: h^2/36 [4 2 2 1]
        np.testing.assert_allclose(M[0], h * h / 36 * np.array([4, 2, 2, 1]), rtol=1e-13)


def test_trilinear_isotropic_closed_form():
    # trilinear-hex Laplacian (unit D): h/3 diagonal, 0 along edges,
    # -h/12 across face diagonals and the body diagonal
    h = 0.02
    K, M = fem.box_element_matrices(3, h, np.eye(3))
    for a in range(8):
        for b in range(8):
            d = bin(a ^ b).count("1")
            expect = {0: 1 / 3, 1: 0.0, 2: -1 / 12, 3: -1 / 12}[d] * h
            assert abs(K[a, b] - expect) < 1e-15
    np.testing.assert_allclose(M.sum(axis=1), np.full(8, h ** 3 / 8), rtol=1e-13)


def test_tet_reference_closed_form():
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=float)
    K, M = fem.tet_element_matrices(X, np.eye(3))
    exp = np.array([[3, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6.0
    np.testing.assert_allclose(K, exp, atol=1e-15)
    np.testing.assert_allclose(M.sum(), 1.0 / 6.0, rtol=1e-14)   # integral of 1 = volume


def test_conductivity_tensor_eigenstructure():
    f = np.array([[math.cos(0.3), math.sin(0.3), 0.0]])
    D = fem.conductivity_tensor([2.0], [0.5], f, 3)[0]
    np.testing.assert_allclose(D @ f[0], 2.0 * f[0], atol=1e-15)
    t = np.array([-math.sin(0.3), math.cos(0.3), 0.0])
    np.testing.assert_allclose(D @ t, 0.5 * t, atol=1e-15)
    np.testing.assert_allclose(D @ np.array([0, 0, 1.0]), [0, 0, 0.5], atol=1e-15)


def _interior(dim, n):
    xyz = I.grid_node_coords(dim, n, 1.0)
    ok = np.ones(len(xyz), bool)
    for d in range(dim):
        ok &= (xyz[:, d] > 0) & (xyz[:, d] < n[d] - 1)
    return ok


@pytest.mark.parametrize("dim", [2, 3])
def test_grid_patch_tests(dim):
    """K 1 = 0; K (linear) = 0 inside; (K quad)_i / m_i = -tr(D B) inside (uniform grid)."""
    wl = I.tp06_slab_3d(7, 6, 5, h=0.1) if dim == 3 else I.aniso_sheet_2d(n=7, length=0.6)
    rng = np.random.default_rng(0)
    ne = wl.n_elems
    ang = 0.7
    fib = np.tile([math.cos(ang), math.sin(ang), 0.0], (ne, 1))
    K, m = fem.assemble_grid(dim, wl.n, wl.h, np.full(ne, 1.3), np.full(ne, 0.4), fib)
    n_nodes = K.shape[0]
    assert abs(K - K.T).max() < 1e-15
    np.testing.assert_allclose(K @ np.ones(n_nodes), 0.0, atol=1e-14)
    xyz = I.grid_node_coords(dim, wl.n, wl.h)[:, :dim]
    inner = _interior(dim, wl.n)
    a = rng.standard_normal(dim)
    np.testing.assert_allclose((K @ (xyz @ a))[inner], 0.0, atol=1e-13)
    B = rng.standard_normal((dim, dim))
    B = B + B.T
    u = 0.5 * np.einsum("ni,ij,nj->n", xyz, B, xyz)
    D = fem.conductivity_tensor([1.3], [0.4], fib[:1], dim)[0]
    np.testing.assert_allclose(((K @ u) / m)[inner], -np.trace(D @ B), rtol=1e-10)
    # lumped mass sums to the domain measure
    L = [(wl.n[d] - 1) * wl.h for d in range(dim)]
    assert abs(m.sum() - np.prod(L)) < 1e-12 * np.prod(L)


def test_tet_patch_tests():
    wl = I.tet_slab_3d(6, 5, 4, h=0.1, fibrosis=0.0, scar_radius=0.0)
    # the linear patch test needs one constant tensor across each node's patch
    fib = np.tile([math.cos(0.4), math.sin(0.4), 0.0], (wl.n_elems, 1))
    K, m = fem.assemble_tets(wl.xyz, wl.tets, wl.d_long, wl.d_trans, fib)
    K2, m2 = fem.assemble_tets_vectorised(wl.xyz, wl.tets, wl.d_long, wl.d_trans, fib)
    assert abs(K - K2).max() < 1e-15 and np.abs(m - m2).max() < 1e-15
    assert abs(K - K.T).max() < 1e-16
    np.testing.assert_allclose(K @ np.ones(K.shape[0]), 0.0, atol=1e-16)
    xyz = wl.xyz
    nx, ny, nz = wl.meta["grid"]
    idx = np.arange(len(xyz))
    ix, iy, iz = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    inner = (ix > 0) & (ix < nx - 1) & (iy > 0) & (iy < ny - 1) & (iz > 0) & (iz < nz - 1)
    u = xyz @ np.array([0.3, -1.1, 0.7])
    np.testing.assert_allclose((K @ u)[inner], 0.0, atol=1e-18)
    assert abs(m.sum() - 0.5 * 0.4 * 0.3) < 1e-14
    # Kuhn split of a regular grid couples each interior node to 14 others
    nnz = np.diff(K.indptr)
    assert (nnz[inner] == 15).all()


def test_isotropic_gershgorin_closed_form():
    # bilinear quads, isotropic D, lumped mass: every row gives 3 h^2 / (16 D)
    wl = I.ms_square_2d()
    K, m = fem.assemble_grid(2, wl.n, wl.h, wl.d_long, wl.d_trans, wl.fibre)
    dt_s = scheme.gershgorin_dt(K, m)
    assert abs(dt_s - 0.9 * 3 * wl.h ** 2 / (16 * 0.001)) < 1e-15
    assert abs(dt_s - 0.10546875) < 1e-15


def test_section31_printed_dt_s():
    g = json.load(open(os.path.join(GOLDEN, "section31_dt_s.json")))
    n = 11
    wl = I.aniso_sheet_2d(n=n, length=(n - 1) * g["h_cm"], d0=g["d0"], rho=g["rho"])
    K, m = fem.assemble_grid(2, wl.n, wl.h, wl.d_long, wl.d_trans, wl.fibre)
    dt_s = scheme.gershgorin_dt(K, m)
    assert round(dt_s, g["printed_digits"]) == g["printed_dt_s_ms"]
    # and the closed form 0.9 h^2 / (4 d0) for rho = 1/4 with fibres along X
    assert abs(dt_s - 0.9 * g["h_cm"] ** 2 / (4 * g["d0"])) < 1e-15


def test_table1_mesh_counts():
    g = json.load(open(os.path.join(GOLDEN, "table1_mesh_counts.json")))
    for row in g["rows"]:
        n_el = int(math.floor(g["side_cm"] / (row["h_um"] * 1e-4) + 1e-9))
        assert n_el * n_el == row["elements"]
        assert (n_el + 1) ** 2 == row["nodes"]
