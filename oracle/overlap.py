"""Dense FP64 overlap construction on small lattices (Sec. 7.1, Eq. def_over
and Eq. def_mass) and the spectra studied in Sec. 7.4.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the product package
never imports it.  Everything here is the plain definition written out with
dense matrices (n = 12 V unknowns, so lattices of a few hundred sites):

  * the matrix of D (the class operator of Sec. 8 with the weights currently
    set in the oracle) is assembled column by column from ``oracle.apply``;
  * sign(H) of the hermitian H = gamma5 (D - rho) is V sign(Lambda) V^dagger
    from a dense hermitian eigendecomposition (numpy ``eigh``);
  * D_ov = rho [1 + gamma5 sign(H)] (Eq. def_over, second form) and the
    massive D_ov,m = (1 - m / (2 rho)) D_ov + m (Eq. def_mass), lattice
    spacing a = 1;
  * the first form of Eq. def_over, rho [1 + X (X^dagger X)^(-1/2)] with
    X = D(m0 = -rho), from an eigendecomposition of X^dagger X;
  * the eigenvalues of A = X^dagger X, whose extremal Ritz values Sec. 7.4
    compares between kernels.

Element order of a vector: [site][spin][colour], sites x0 fastest, the same as
``oracle.apply``.  Pinned by tests/test_oracle_overlap.py (free-field
momentum-space form, Ginsparg-Wilson relation, normality, the circle of
Eq. def_mass, agreement of the two forms of Eq. def_over).
"""
import numpy as np

import oracle


def _volume(L):
    return int(np.prod(L))


def dirac_matrix(L, bc, W, m0, dagger=False):
    """Dense (12V, 12V) matrix of D(m0) (or D^dagger) from unit-vector columns."""
    V = _volume(L)
    n = 12 * V
    M = np.zeros((n, n), np.complex128)
    e = np.zeros((V, 4, 3), np.complex128)
    for j in range(n):
        e.reshape(-1)[j] = 1.0
        M[:, j] = oracle.apply(L, bc, W, m0, e, dagger=dagger).reshape(-1)
        e.reshape(-1)[j] = 0.0
    return M


def gamma5_matrix(L):
    """gamma5 acting on every site, colour unchanged."""
    return np.kron(np.eye(_volume(L)), np.kron(oracle.gamma(4), np.eye(3)))


def hermitian_kernel(L, bc, W, rho=1.0):
    """H = gamma5 (D - rho) (Sec. 7.4: the shifted hermitian kernel)."""
    return gamma5_matrix(L) @ dirac_matrix(L, bc, W, -rho)


def sign_hermitian(H):
    """sign(H) = V sign(Lambda) V^dagger for hermitian H (no zero eigenvalue)."""
    lam, Q = np.linalg.eigh(H)
    if np.min(np.abs(lam)) == 0.0:
        raise ValueError("H has an exact zero mode; sign(H) is undefined")
    return (Q * np.sign(lam)) @ Q.conj().T


def overlap_matrix(L, bc, W, rho=1.0, m=0.0):
    """D_ov,m = (1 - m/(2 rho)) rho [1 + gamma5 sign(gamma5 (D - rho))] + m."""
    G5 = gamma5_matrix(L)
    S = sign_hermitian(hermitian_kernel(L, bc, W, rho))
    n = S.shape[0]
    Dov = rho * (np.eye(n) + G5 @ S)
    return (1.0 - m / (2.0 * rho)) * Dov + m * np.eye(n)


def overlap_matrix_invsqrt(L, bc, W, rho=1.0):
    """First form of Eq. def_over: rho [1 + X (X^dagger X)^(-1/2)], X = D(-rho)."""
    X = dirac_matrix(L, bc, W, -rho)
    mu, Q = np.linalg.eigh(X.conj().T @ X)
    inv_sqrt = (Q / np.sqrt(mu)) @ Q.conj().T
    return rho * (np.eye(X.shape[0]) + X @ inv_sqrt)


def ddag_d_eigenvalues(L, bc, W, m0):
    """Ascending eigenvalues of A = D(m0)^dagger D(m0)."""
    D = dirac_matrix(L, bc, W, m0)
    return np.linalg.eigvalsh(D.conj().T @ D)


def kernel_eigenpairs(L, bc, W, rho=1.0):
    """Eigenvalues (ascending |lambda|) and eigenvectors (columns) of H."""
    lam, Q = np.linalg.eigh(hermitian_kernel(L, bc, W, rho))
    order = np.argsort(np.abs(lam), kind="stable")
    return lam[order], Q[:, order]
