"""Synthetic finite-element pencils (A, B) that stand in for the paper's vibration models.

The paper's meshes (Pyramid S1/S2, hollow platform, fish-like; Section 3.1) are not
available, so every workload is assembled here from structured grids:

* ``bar1d``            - 1D linear-FEM bar, Dirichlet at both ends.
* ``q1_scalar``        - Q1 (bi/trilinear) scalar Laplacian + consistent mass on a
                          2D or 3D box grid, optional per-element coefficient,
                          optional Dirichlet face, optional ``+shift*B``.
* ``q1_elasticity``    - Q1 linear elasticity, 3 dof/node, 2x2x2 Gauss quadrature,
                          per-element Young's modulus, one clamped face (the paper's
                          governing equation, Section 3.1, with Dirichlet part Gamma_D).

All matrices are returned as one shared CSR pattern with two FP64 value arrays, the
layout the solver library consumes: ``rowptr`` int64[n+1], ``col`` int32[nnz] (sorted
within each row), ``valA`` / ``valB`` float64[nnz].  Both matrices are assembled over
the same element connectivity, so their patterns are identical by construction.

This module is input generation only: it contains none of the eigensolver's arithmetic.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class CsrPair:
    """Two symmetric matrices over one CSR pattern."""

    n: int
    rowptr: np.ndarray  # int64[n+1]
    col: np.ndarray  # int32[nnz]
    valA: np.ndarray  # float64[nnz]
    valB: np.ndarray  # float64[nnz]

    @property
    def nnz(self) -> int:
        return int(self.col.shape[0])

    def A(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.valA, self.col, self.rowptr), shape=(self.n, self.n))

    def B(self) -> sp.csr_matrix:
        return sp.csr_matrix((self.valB, self.col, self.rowptr), shape=(self.n, self.n))


def _pair_from_coo(rows, cols, va, vb, n, keep=None) -> CsrPair:
    """Sum duplicates of two COO value lists on identical coordinates into one pattern."""
    A = sp.coo_matrix((va, (rows, cols)), shape=(n, n)).tocsr()
    B = sp.coo_matrix((vb, (rows, cols)), shape=(n, n)).tocsr()
    if keep is not None:
        A = A[keep][:, keep].tocsr()
        B = B[keep][:, keep].tocsr()
    A.sort_indices()
    B.sort_indices()
    if not (np.array_equal(A.indptr, B.indptr) and np.array_equal(A.indices, B.indices)):
        raise RuntimeError("A and B patterns differ")
    return CsrPair(
        n=A.shape[0],
        rowptr=A.indptr.astype(np.int64),
        col=A.indices.astype(np.int32),
        valA=np.ascontiguousarray(A.data, dtype=np.float64),
        valB=np.ascontiguousarray(B.data, dtype=np.float64),
    )


def bar1d(n: int) -> CsrPair:
    """1D linear-FEM bar on (0,1), n interior nodes, h = 1/(n+1), Dirichlet ends.

    Stiffness tridiag(-1, 2, -1)/h, consistent mass h/6 * tridiag(1, 4, 1).
    """
    h = 1.0 / (n + 1)
    i = np.arange(n)
    rows = np.concatenate([i, i[1:], i[:-1]])
    cols = np.concatenate([i, i[:-1], i[1:]])
    va = np.concatenate([np.full(n, 2.0 / h), np.full(n - 1, -1.0 / h), np.full(n - 1, -1.0 / h)])
    vb = np.concatenate([np.full(n, 4.0 * h / 6.0), np.full(n - 1, h / 6.0), np.full(n - 1, h / 6.0)])
    return _pair_from_coo(rows, cols, va, vb, n)


def _k1(h):
    return np.array([[1.0, -1.0], [-1.0, 1.0]]) / h


def _m1(h):
    return np.array([[2.0, 1.0], [1.0, 2.0]]) * h / 6.0


def _grid_connectivity(shape_nodes):
    """Element -> node map for a structured grid, lexicographic numbering (x fastest).

    Local node l of an element has offsets (a, b[, c]) with l = a + 2b (+ 4c).
    """
    dim = len(shape_nodes)
    ne = [s - 1 for s in shape_nodes]
    idx = np.indices(ne).reshape(dim, -1)  # idx[d] = element coordinate along axis d
    strides = np.cumprod([1] + list(shape_nodes[:-1]))
    base = sum(idx[d] * strides[d] for d in range(dim))
    offs = []
    for l in range(2**dim):
        bits = [(l >> d) & 1 for d in range(dim)]
        offs.append(sum(bits[d] * strides[d] for d in range(dim)))
    # np.indices iterates axis 0 slowest; order elements so that the x index is fastest
    order = np.lexsort(tuple(idx[d] for d in range(dim)))
    base = base[order]
    return base[:, None] + np.array(offs)[None, :], order


def q1_scalar(nodes, coef=None, shift=0.0, dirichlet_face=None, lengths=None) -> CsrPair:
    """Q1 scalar Laplacian and consistent mass on a 2D/3D box.

    ``nodes`` = (nx, ny[, nz]) grid nodes; ``coef`` per-element stiffness coefficient
    (x-fastest element order) or None for 1; ``shift`` adds shift*B to A; ``dirichlet_face``
    = (axis, 0|1) removes the nodes on that face.  Element matrices are the exact
    tensor products of the 1D linear element matrices.
    """
    nodes = tuple(int(s) for s in nodes)
    dim = len(nodes)
    if lengths is None:
        lengths = (1.0,) * dim
    hs = [lengths[d] / (nodes[d] - 1) for d in range(dim)]
    ks = [_k1(h) for h in hs]
    ms = [_m1(h) for h in hs]
    # local index l = a + 2b + 4c  ->  kron(z, kron(y, x))
    if dim == 2:
        Ke = np.kron(ms[1], ks[0]) + np.kron(ks[1], ms[0])
        Me = np.kron(ms[1], ms[0])
    elif dim == 3:
        Ke = (np.kron(ms[2], np.kron(ms[1], ks[0])) + np.kron(ms[2], np.kron(ks[1], ms[0]))
              + np.kron(ks[2], np.kron(ms[1], ms[0])))
        Me = np.kron(ms[2], np.kron(ms[1], ms[0]))
    else:
        raise ValueError("dim must be 2 or 3")
    conn, _ = _grid_connectivity(nodes)
    ne = conn.shape[0]
    c = np.ones(ne) if coef is None else np.asarray(coef, dtype=np.float64).reshape(ne)
    nl = conn.shape[1]
    rows = np.repeat(conn, nl, axis=1).ravel()
    cols = np.tile(conn, (1, nl)).ravel()
    va = (c[:, None] * Ke.ravel()[None, :] + shift * Me.ravel()[None, :]).ravel()
    vb = np.broadcast_to(Me.ravel()[None, :], (ne, nl * nl)).ravel()
    n = int(np.prod(nodes))
    keep = None
    if dirichlet_face is not None:
        axis, side = dirichlet_face
        coords = np.indices(nodes[::-1]).reshape(dim, -1)[::-1]  # coords[d] of node id (x fastest)
        bnd = coords[axis] == (0 if side == 0 else nodes[axis] - 1)
        keep = np.nonzero(~bnd)[0]
    return _pair_from_coo(rows, cols, va, vb, n, keep)


def _elasticity_element(h, nu):
    """24x24 stiffness (unit Young's modulus) and consistent mass (unit density) of a
    cube element of side h, trilinear shape functions, 2x2x2 Gauss quadrature.

    DOF ordering 3*l + component, l = a + 2b + 4c.
    """
    lam = nu / ((1 + nu) * (1 - 2 * nu))
    mu = 1.0 / (2 * (1 + nu))
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[3, 3] = D[4, 4] = D[5, 5] = mu
    g = np.array([-1.0, 1.0]) / np.sqrt(3.0)
    signs = np.array([[(l >> d) & 1 for d in range(3)] for l in range(8)]) * 2 - 1  # +-1
    K = np.zeros((24, 24))
    M = np.zeros((24, 24))
    jac = (h / 2.0) ** 3
    for xi in g:
        for eta in g:
            for zeta in g:
                q = np.array([xi, eta, zeta])
                N = np.prod(1 + signs * q[None, :], axis=1) / 8.0
                dN = np.zeros((8, 3))
                for d in range(3):
                    other = [e for e in range(3) if e != d]
                    dN[:, d] = signs[:, d] * np.prod(1 + signs[:, other] * q[None, other], axis=1) / 8.0
                dN *= 2.0 / h  # d/dx = (2/h) d/dxi
                Bm = np.zeros((6, 24))
                for l in range(8):
                    dx, dy, dz = dN[l]
                    Bm[:, 3 * l:3 * l + 3] = [[dx, 0, 0], [0, dy, 0], [0, 0, dz],
                                              [dy, dx, 0], [0, dz, dy], [dz, 0, dx]]
                K += Bm.T @ D @ Bm * jac
                M += np.kron(np.outer(N, N), np.eye(3)) * jac
    return K, M


def q1_elasticity(nodes, E=None, nu=0.3, rho=1.0, clamp_face=(2, 0), length=None) -> CsrPair:
    """3D Q1 linear elasticity, 3 dof/node on an (nx, ny, nz)-node box of cubes.

    ``E`` per-element Young's modulus (x-fastest element order) or None for 1;
    ``clamp_face`` = (axis, side) fixes every dof on that face (default z = 0).
    The element size is h = 1/(max(nodes) - 1) unless ``length`` (of the longest edge) is given.
    """
    nodes = tuple(int(s) for s in nodes)
    h = (1.0 if length is None else float(length)) / (max(nodes) - 1)
    Ke, Me = _elasticity_element(h, nu)
    Me = rho * Me
    conn, _ = _grid_connectivity(nodes)
    ne = conn.shape[0]
    dofs = (3 * conn[:, :, None] + np.arange(3)[None, None, :]).reshape(ne, 24)
    Ev = np.ones(ne) if E is None else np.asarray(E, dtype=np.float64).reshape(ne)
    rows = np.repeat(dofs, 24, axis=1).ravel()
    cols = np.tile(dofs, (1, 24)).ravel()
    va = (Ev[:, None] * Ke.ravel()[None, :]).ravel()
    vb = np.broadcast_to(Me.ravel()[None, :], (ne, 576)).ravel()
    nnodes = int(np.prod(nodes))
    keep = None
    if clamp_face is not None:
        axis, side = clamp_face
        coords = np.indices(nodes[::-1]).reshape(3, -1)[::-1]
        bnd = coords[axis] == (0 if side == 0 else nodes[axis] - 1)
        free_nodes = np.nonzero(~bnd)[0]
        keep = (3 * free_nodes[:, None] + np.arange(3)[None, :]).ravel()
    return _pair_from_coo(rows, cols, va, vb, 3 * nnodes, keep)
