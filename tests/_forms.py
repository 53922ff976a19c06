"""Independent mathematical forms used to pin the oracle (test helpers).

Nothing here reuses the oracle's loops: the smoothers are written as sparse
matrix operators (scipy.sparse Kronecker sums) and the closed forms of the
discrete sine modes.  Interior vectors are flattened in C order (k, j, i).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def tridiag_ones(n: int) -> sp.csr_matrix:
    """n x n matrix with ones on the first off-diagonals (1D neighbour sum)."""
    if n == 1:
        return sp.csr_matrix((1, 1))
    off = np.ones(n - 1)
    return sp.diags([off, off], [-1, 1], format="csr")


def neighbour_matrix(nx: int, ny: int, nz: int) -> sp.csr_matrix:
    """Sum of the six interior neighbours as a sparse matrix (Kronecker sum)."""
    ix, iy, iz = sp.identity(nx), sp.identity(ny), sp.identity(nz)
    return (sp.kron(sp.kron(iz, iy), tridiag_ones(nx))
            + sp.kron(sp.kron(iz, tridiag_ones(ny)), ix)
            + sp.kron(sp.kron(tridiag_ones(nz), iy), ix)).tocsr()


def lex_split(nx: int, ny: int, nz: int):
    """(L, U): neighbours earlier / later in lexicographic (k, j, i) order."""
    n = neighbour_matrix(nx, ny, nz)
    return sp.tril(n, k=-1).tocsr(), sp.triu(n, k=1).tocsr()


def boundary_sum(u: np.ndarray) -> np.ndarray:
    """Per interior site, the sum of its neighbours that lie in the halo."""
    nz, ny, nx = (s - 2 for s in u.shape)
    b = np.zeros((nz, ny, nx))
    b[:, :, 0] += u[1:-1, 1:-1, 0]
    b[:, :, -1] += u[1:-1, 1:-1, -1]
    b[:, 0, :] += u[1:-1, 0, 1:-1]
    b[:, -1, :] += u[1:-1, -1, 1:-1]
    b[0, :, :] += u[0, 1:-1, 1:-1]
    b[-1, :, :] += u[-1, 1:-1, 1:-1]
    return b.ravel()


def interior(u: np.ndarray) -> np.ndarray:
    return np.array(u[1:-1, 1:-1, 1:-1], dtype=np.float64).ravel()


def sine_mode(nx: int, ny: int, nz: int, p: int, q: int, r: int) -> np.ndarray:
    """Padded array holding sin(p pi x/(nx+1)) sin(q pi y/(ny+1)) sin(r pi z/(nz+1))
    at the 1-based interior coordinates, exactly zero on the halo."""
    x = np.sin(p * np.pi * np.arange(1, nx + 1) / (nx + 1))
    y = np.sin(q * np.pi * np.arange(1, ny + 1) / (ny + 1))
    z = np.sin(r * np.pi * np.arange(1, nz + 1) / (nz + 1))
    u = np.zeros((nz + 2, ny + 2, nx + 2))
    u[1:-1, 1:-1, 1:-1] = z[:, None, None] * y[None, :, None] * x[None, None, :]
    return u


def jacobi_factor(nx, ny, nz, p, q, r) -> float:
    """One Jacobi sweep (a=0, b=1/6, f=0) multiplies the (p,q,r) mode by this."""
    return (np.cos(p * np.pi / (nx + 1)) + np.cos(q * np.pi / (ny + 1)) + np.cos(r * np.pi / (nz + 1))) / 3.0


def eigenvalue(nx, ny, nz, p, q, r, h) -> float:
    """A = (6 I - neighbour sum)/h^2 applied to the (p,q,r) mode multiplies it by this."""
    return (6.0 - 2 * np.cos(p * np.pi / (nx + 1)) - 2 * np.cos(q * np.pi / (ny + 1))
            - 2 * np.cos(r * np.pi / (nz + 1))) / (h * h)


def harmonic_fields(nx: int, ny: int, nz: int):
    """Polynomials whose 7-point discrete Laplacian is zero, evaluated at the padded
    integer coordinates (halo included)."""
    z, y, x = np.meshgrid(np.arange(nz + 2, dtype=np.float64), np.arange(ny + 2, dtype=np.float64),
                          np.arange(nx + 2, dtype=np.float64), indexing="ij")
    return {
        "x+2y-3z": x + 2 * y - 3 * z,
        "xy+yz+zx": x * y + y * z + z * x,
        "x2-y2": x * x - y * y,
        "xyz": x * y * z,
        "x2+y2-2z2": x * x + y * y - 2 * z * z,
    }
