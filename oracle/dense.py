"""Dense brute-force references, used only to pin the oracle (test infrastructure only).

Sizes are tiny (8 x 8, 4 x 4 x 4); everything is an explicit matrix.
"""
from __future__ import annotations

import itertools

import numpy as np


def dft_matrix(N):
    """F_jk = exp(-2 pi i j k / N) (unnormalised forward DFT)."""
    j = np.arange(N)
    return np.exp(-2j * np.pi * np.outer(j, j) / N)


def dense_dftn(x):
    """n-dimensional DFT of a real/complex array by successive dense matrix products."""
    out = np.asarray(x, dtype=complex)
    for ax in range(out.ndim):
        F = dft_matrix(out.shape[ax])
        out = np.moveaxis(np.tensordot(F, np.moveaxis(out, ax, 0), axes=(1, 0)), 0, ax)
    return out


def _lin(shape, idx):
    return int(np.ravel_multi_index(tuple(i % s for i, s in zip(idx, shape)), shape))


def rotated_gradient_matrix(shape):
    """Real-space gradient of the rotated scheme (Willot): nodal displacements at the voxel
    corners p + 1/2, strain at voxel centres; the derivative along a at voxel v is the
    average over the 2^(d-1) cell edges parallel to a of the nodal differences.

    Returns D of shape (d*d*n, d*n) mapping u[b, node] to grad[a, b, voxel] = d u_b / d x_a.
    Array axis order of the grid is [.., y, x]; direction a = 0 is x (last axis).
    """
    d = len(shape)
    n = int(np.prod(shape))
    D = np.zeros((d, d, n, d, n))
    for v in itertools.product(*[range(s) for s in shape]):
        vi = _lin(shape, v)
        for a in range(d):
            ax = d - 1 - a
            others = [b for b in range(d) if b != a]
            for bits in itertools.product((0, 1), repeat=d - 1):
                s = [0] * d  # shift per array axis (1 = node at v - 1 along that axis)
                for b, bit in zip(others, bits):
                    s[d - 1 - b] = bit
                hi = tuple(v[k] - s[k] for k in range(d))
                lo = list(hi)
                lo[ax] -= 1
                wgt = 1.0 / 2 ** (d - 1)
                for comp in range(d):
                    D[a, comp, vi, comp, _lin(shape, hi)] += wgt
                    D[a, comp, vi, comp, _lin(shape, tuple(lo))] -= wgt
    return D.reshape(d * d * n, d * n)


def spectral_derivative_1d(N, nyquist="zero"):
    """Dense real N x N matrix of the spectral derivative (1/N) F^H diag(s) F along one
    periodic axis, s = i xi with xi = 2 pi k / N; at the Nyquist index (even N) s = 0
    (nyquist="zero") or the real multiplier |xi| = pi (nyquist="real")."""
    F = dft_matrix(N)
    k = np.arange(N)
    ks = np.where(2 * k < N, k, k - N)
    xi = 2.0 * np.pi * ks / N
    s = 1j * xi
    if N % 2 == 0:
        s[N // 2] = 0.0 if nyquist == "zero" else np.pi
    M = (F.conj().T @ np.diag(s) @ F) / N
    return M.real


def spectral_gradient_matrix(shape):
    """Spectral gradient on the voxel grid: D of shape (d*d*n, d*n) mapping u[b, voxel] to
    grad[a, b, voxel] = d u_b / d x_a, built from dense 1D derivative matrices (Kronecker
    products over the array axes [.., y, x]; direction a = 0 is x)."""
    d = len(shape)
    n = int(np.prod(shape))
    D = np.zeros((d, d, n, d, n))
    for a in range(d):
        ax = d - 1 - a
        mats = [np.eye(s) for s in shape]
        mats[ax] = spectral_derivative_1d(shape[ax])
        K = mats[0]
        for m in mats[1:]:
            K = np.kron(K, m)
        for comp in range(d):
            D[a, comp, :, comp, :] = K
    return D.reshape(d * d * n, d * n)


def sym_strain_matrix(shape, scheme="rotated"):
    """B = sym(grad) of the rotated scheme (or of the spectral derivative, scheme =
    "spectral"): (d*d*n) x (d*n), output ordered [i, j, voxel]."""
    d = len(shape)
    n = int(np.prod(shape))
    G = rotated_gradient_matrix(shape) if scheme == "rotated" else spectral_gradient_matrix(shape)
    D = G.reshape(d, d, n, d * n)
    B = 0.5 * (D + np.swapaxes(D, 0, 1))
    return B.reshape(d * d * n, d * n)


def compatible_projector(shape, scheme="rotated"):
    """Orthogonal projector (Frobenius metric) onto the range of B: P = B B^+."""
    B = sym_strain_matrix(shape, scheme)
    return B @ np.linalg.pinv(B, rcond=1e-10)


def field_to_vec(tau):
    """(shape + (d, d)) -> vector ordered [i, j, voxel]."""
    d = tau.shape[-1]
    return np.moveaxis(tau.reshape(-1, d, d), 0, -1).reshape(-1)


def vec_to_field(v, shape):
    d = len(shape)
    return np.moveaxis(v.reshape(d, d, -1), -1, 0).reshape(tuple(shape) + (d, d))


def sym_basis(d):
    """Orthonormal basis of symmetric d x d tensors (Frobenius): e_i e_i and (e_i e_j + e_j e_i)/sqrt 2."""
    out = []
    for i in range(d):
        for j in range(i, d):
            T = np.zeros((d, d))
            if i == j:
                T[i, i] = 1.0
            else:
                T[i, j] = T[j, i] = 1.0 / np.sqrt(2.0)
            out.append(T)
    return out


def dense_jacobian(apply, shape, d):
    """Columns of the Jacobian in the orthonormal symmetric basis: unknown ordering
    [voxel-major sym components (m*n), phi (n), E (1)]; rows use the same basis."""
    basis = sym_basis(d)
    m = len(basis)
    n = int(np.prod(shape))
    N = m * n + n + 1

    def pack(v):
        e, p, E = v
        ef = e.reshape(n, d, d)
        comps = np.stack([np.einsum("vij,ij->v", ef, T) for T in basis], axis=1).reshape(-1)
        return np.concatenate([comps, p.reshape(-1), [E]])

    J = np.zeros((N, N))
    for c in range(N):
        e = np.zeros((n, d, d))
        p = np.zeros(n)
        E = 0.0
        if c < m * n:
            e[c // m] = basis[c % m]
        elif c < m * n + n:
            p[c - m * n] = 1.0
        else:
            E = 1.0
        J[:, c] = pack(apply((e.reshape(tuple(shape) + (d, d)), p.reshape(shape), E)))
    return J, pack


def compatible_basis_sym(shape):
    """Orthonormal basis (columns) of compatible symmetric strain fields, in the packing of
    ``dense_jacobian`` (voxel-major, symmetric components in ``sym_basis`` order)."""
    d = len(shape)
    n = int(np.prod(shape))
    B = sym_strain_matrix(shape).reshape(d, d, n, d * n)
    basis = sym_basis(d)
    m = len(basis)
    Bs = np.zeros((n, m, d * n))
    for c, T in enumerate(basis):
        Bs[:, c, :] = np.einsum("ij,ijvk->vk", T, B)
    Bs = Bs.reshape(n * m, d * n)
    U, s, _ = np.linalg.svd(Bs, full_matrices=False)
    return U[:, s > 1e-10 * s[0]]


def restricted_solver(shape, d):
    """Dense linear solver for the oracle's Newton loop: solves J x = b exactly with x
    restricted to compatible strains (+ all phi, E), by least squares on J Q."""
    Qc = compatible_basis_sym(shape)
    n = int(np.prod(shape))
    mn = Qc.shape[0]
    r = Qc.shape[1]
    Q = np.zeros((mn + n + 1, r + n + 1))
    Q[:mn, :r] = Qc
    Q[mn:, r:] = np.eye(n + 1)
    basis = sym_basis(d)
    m = len(basis)

    def solve(lin, A, b, control):
        J, pack = dense_jacobian(A, shape, d)
        rhs = pack(b)
        y, *_ = np.linalg.lstsq(J @ Q, rhs, rcond=None)
        x = Q @ y
        comps = x[:mn].reshape(n, m)
        e = np.einsum("vc,cij->vij", comps, np.stack(basis)).reshape(tuple(shape) + (d, d))
        sol = (e, x[mn:mn + n].reshape(shape), float(x[-1]))
        res = np.linalg.norm(J @ x - rhs) / max(np.linalg.norm(rhs), 1e-300)
        return sol, 1, res, 0

    return solve
