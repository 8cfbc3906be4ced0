"""Seeded synthetic inputs shared by the oracle and the CUDA-path tests.

This module only draws random numbers and assembles matrices by plain matrix
products; it holds none of the method's arithmetic (no drift, no cooling, no
exponential of a Lie-algebra element, no determinant re-projection).

* SU(3) matrices are products of random SU(2) rotations embedded in the three
  2x2 blocks (each block is a unit quaternion, so det = 1 and U U^+ = 1).
* SL(3,C) matrices multiply such an SU(3) matrix by a lower unipotent matrix,
  a diagonal matrix diag(a, b, 1/(ab)) and an upper unipotent matrix, each of
  determinant exactly one; `spread` sets how far the result is from SU(3).
* The constant-flux configuration is an abelian field with a known plaquette
  angle in every plane, the input of the closed-form pins.
"""
import numpy as np


def rng(seed):
    return np.random.default_rng(seed)


def _su2_block(r, n, i, j):
    q = r.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    a0, a1, a2, a3 = q.T
    M = np.zeros((n, 3, 3), np.complex128)
    M[:] = np.eye(3)
    M[:, i, i] = a0 + 1j * a3
    M[:, i, j] = a2 + 1j * a1
    M[:, j, i] = -a2 + 1j * a1
    M[:, j, j] = a0 - 1j * a3
    return M


def random_su3(r, n):
    """n random SU(3) matrices (shape (n,3,3))."""
    M = np.broadcast_to(np.eye(3, dtype=np.complex128), (n, 3, 3)).copy()
    for _ in range(2):
        for (i, j) in ((0, 1), (0, 2), (1, 2)):
            M = M @ _su2_block(r, n, i, j)
    return M


def random_sl3c(r, n, spread=0.3):
    """n random SL(3,C) matrices, `spread` away from SU(3)."""
    low = np.broadcast_to(np.eye(3, dtype=np.complex128), (n, 3, 3)).copy()
    up = low.copy()
    z = lambda: spread * (r.normal(size=n) + 1j * r.normal(size=n))
    low[:, 1, 0], low[:, 2, 0], low[:, 2, 1] = z(), z(), z()
    up[:, 0, 1], up[:, 0, 2], up[:, 1, 2] = z(), z(), z()
    a = np.exp(z())
    b = np.exp(z())
    D = np.zeros((n, 3, 3), np.complex128)
    D[:, 0, 0], D[:, 1, 1], D[:, 2, 2] = a, b, 1.0 / (a * b)
    return random_su3(r, n) @ low @ D @ up


def volume(L):
    return int(np.prod(L))


def su3_lattice(L, seed):
    r = rng(seed)
    return random_su3(r, 4 * volume(L)).reshape(volume(L), 4, 3, 3)


def sl3c_lattice(L, seed, spread=0.3):
    r = rng(seed)
    return random_sl3c(r, 4 * volume(L), spread).reshape(volume(L), 4, 3, 3)


def sl3c_sites(L, seed, spread=0.3):
    """One SL(3,C) matrix per site (a gauge transformation)."""
    r = rng(seed)
    return random_sl3c(r, volume(L), spread)


def coords(L):
    """Integer coordinates of every site, shape (V,4), site s = x0 + L0*(x1 + ...)."""
    V = volume(L)
    s = np.arange(V)
    x = np.zeros((V, 4), np.int64)
    for mu in range(4):
        x[:, mu] = s % L[mu]
        s = s // L[mu]
    return x


def constant_flux(L, n):
    """Abelian links U = diag(e^{iA}, e^{-iA}, 1) with plaquette angle
    phi_{mu nu} = 2 pi n[mu][nu] / (L_mu L_nu) in every plaquette of plane mu<nu.
    Plane (mu,nu): A_nu(x) += phi x_mu; A_mu(x) -= phi L_mu x_nu where x_mu = L_mu - 1."""
    x = coords(L)
    V = volume(L)
    A = np.zeros((V, 4))
    for mu in range(4):
        for nu in range(mu + 1, 4):
            k = n.get((mu, nu), 0)
            if not k:
                continue
            phi = 2 * np.pi * k / (L[mu] * L[nu])
            A[:, nu] += phi * x[:, mu]
            edge = x[:, mu] == L[mu] - 1
            A[edge, mu] -= phi * L[mu] * x[edge, nu]
    U = np.zeros((V, 4, 3, 3), np.complex128)
    U[:, :, 0, 0] = np.exp(1j * A)
    U[:, :, 1, 1] = np.exp(-1j * A)
    U[:, :, 2, 2] = 1.0
    return U


def flux_angles(L, n):
    return {(mu, nu): 2 * np.pi * n.get((mu, nu), 0) / (L[mu] * L[nu])
            for mu in range(4) for nu in range(mu + 1, 4)}


def sample_links(V, k, seed):
    """k distinct link ids (site*4 + mu) drawn uniformly."""
    r = rng(seed)
    return np.sort(r.choice(4 * V, size=min(k, 4 * V), replace=False)).astype(np.int64)
