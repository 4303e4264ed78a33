"""Q1 finite element space on a rectangle and its simultaneous diagonalisation.

Test infrastructure only (see ``oracle/__init__``).

Sec. 2.1 (tensor FE space V_h, weak form with a(w,v) = int D grad w . grad v,
L_h defined by a(w,v) = (L_h w, v)) and the closing paragraph of Sec. 2.3
(mass and stiffness matrices diagonalised at once by one orthogonal matrix,
applied by tensor products).

Conventions: axis a has n_a interior nodes x_k = lo_a + k h_a, k = 1..n_a,
h_a = (hi_a - lo_a)/(n_a + 1) (the paper's N_a subintervals are n_a + 1); a periodic
axis has n_a nodes x_k = lo_a + k h_a, k = 0..n_a - 1, h_a = (hi_a - lo_a)/n_a, and the
discrete Hartley transform takes the place of the DST-I.
Nodal and modal arrays are C-ordered with shape (n_0, ..., n_{d-1}).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg
import scipy.sparse as sp


def axis_grid(lo: float, hi: float, n: int, periodic: bool = False):
    """Mesh size and node coordinates of one axis: n interior nodes x_k = lo + k h, k = 1..n,
    h = (hi - lo)/(n + 1) (Dirichlet), or n nodes x_k = lo + k h, k = 0..n-1, h = (hi - lo)/n
    on a periodic axis (node n is node 0)."""
    if periodic:
        h = (hi - lo) / n
        return h, lo + h * np.arange(0, n, dtype=np.float64)
    h = (hi - lo) / (n + 1)
    x = lo + h * np.arange(1, n + 1, dtype=np.float64)
    return h, x


def mass_1d_periodic(n: int, h: float) -> np.ndarray:
    """1D P1 mass matrix of a periodic axis: circulant (h/6)[1 4 1]."""
    A = 4.0 * np.eye(n)
    for k in range(n):
        A[k, (k + 1) % n] += 1.0
        A[k, (k - 1) % n] += 1.0
    return (h / 6.0) * A


def stiffness_1d_periodic(n: int, h: float) -> np.ndarray:
    """1D P1 stiffness matrix of a periodic axis: circulant (1/h)[-1 2 -1]."""
    A = 2.0 * np.eye(n)
    for k in range(n):
        A[k, (k + 1) % n] -= 1.0
        A[k, (k - 1) % n] -= 1.0
    return A / h


def dht_matrix(n: int) -> np.ndarray:
    """Orthonormal discrete Hartley transform: H[k, j] = (cos + sin)(2 pi j k / n) / sqrt(n).

    Symmetric with H @ H = I; every circulant symmetric matrix is diagonal in it (the
    cosine and sine vectors of one frequency share an eigenvalue).  j k is reduced modulo n.
    """
    k = np.arange(n, dtype=np.int64)
    m = np.outer(k, k) % n
    ang = 2.0 * np.pi * m.astype(np.float64) / n
    return (np.cos(ang) + np.sin(ang)) / np.sqrt(n)


def axis_eigenvalues_periodic(n: int, h: float):
    """Eigenvalues of the periodic 1D mass and stiffness matrices in the DHT basis:
    theta_j = 2 pi j / n, j = 0..n-1, mu^M = (h/3)(2 + cos theta), mu^K = (4/h) sin^2(theta/2)."""
    theta = 2.0 * np.pi * np.arange(n, dtype=np.float64) / n
    return (h / 3.0) * (2.0 + np.cos(theta)), (4.0 / h) * np.sin(0.5 * theta) ** 2


def mass_1d(n: int, h: float) -> np.ndarray:
    """1D P1 mass matrix on interior nodes: (h/6) tridiag(1, 4, 1)."""
    return (h / 6.0) * (4.0 * np.eye(n) + np.eye(n, k=1) + np.eye(n, k=-1))


def stiffness_1d(n: int, h: float) -> np.ndarray:
    """1D P1 stiffness matrix on interior nodes: (1/h) tridiag(-1, 2, -1)."""
    return (1.0 / h) * (2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1))


def assemble(n, box, D, periodic=()):
    """Q1 mass M = kron_a M_a and stiffness K = D sum_a M_1 x .. K_a .. x M_d.

    Returned as scipy sparse CSR matrices acting on C-ordered nodal vectors
    (axis d-1 fastest), i.e. kron(A_0, kron(A_1, ...)).  periodic[a] selects the
    circulant matrices of a periodic axis.
    """
    d = len(n)
    per = tuple(periodic) + (False,) * (d - len(periodic))
    Ms, Ks = [], []
    for a in range(d):
        h, _ = axis_grid(box[a][0], box[a][1], n[a], per[a])
        if per[a]:
            Ms.append(sp.csr_matrix(mass_1d_periodic(n[a], h)))
            Ks.append(sp.csr_matrix(stiffness_1d_periodic(n[a], h)))
        else:
            Ms.append(sp.csr_matrix(mass_1d(n[a], h)))
            Ks.append(sp.csr_matrix(stiffness_1d(n[a], h)))

    def kron_all(mats):
        out = mats[0]
        for m in mats[1:]:
            out = sp.kron(out, m, format="csr")
        return out

    M = kron_all(Ms)
    K = None
    for a in range(d):
        mats = [Ks[b] if b == a else Ms[b] for b in range(d)]
        term = kron_all(mats)
        K = term if K is None else K + term
    return M.tocsr(), (D * K).tocsr()


def dst1_matrix(n: int) -> np.ndarray:
    """Orthonormal DST-I: S[k-1, j-1] = sqrt(2/(n+1)) sin(j k pi/(n+1)).

    S is symmetric and S @ S = I.  The integer j*k is reduced modulo 2(n+1)
    (the period of the sine in that index) before it is scaled by pi/(n+1),
    so every argument lies in [0, 2 pi) and carries no large rounding error.
    """
    k = np.arange(1, n + 1, dtype=np.int64)
    m = np.outer(k, k) % (2 * (n + 1))
    return np.sqrt(2.0 / (n + 1)) * np.sin(m.astype(np.float64) * np.pi / (n + 1))


def axis_eigenvalues(n: int, h: float):
    """Closed-form eigenvalues of the 1D mass and stiffness matrices in the DST-I basis.

    With theta_j = j pi/(n+1):  mu^M_j = (h/3)(2 + cos theta_j),
    mu^K_j = (2/h)(1 - cos theta_j) = (4/h) sin^2(theta_j/2), so that
    S M_a S = diag(mu^M), S K_a S = diag(mu^K).  mu^K is evaluated in the
    sin^2 form, which keeps full relative precision for the slow modes
    (1 - cos theta_1 cancels to ~1e-12 relative at n = 255).
    """
    theta = np.arange(1, n + 1, dtype=np.float64) * np.pi / (n + 1)
    muM = (h / 3.0) * (2.0 + np.cos(theta))
    muK = (4.0 / h) * np.sin(0.5 * theta) ** 2
    return muM, muK


def outer_all(vecs):
    """Tensor (outer) product of 1D arrays -> array of shape (len(v0), len(v1), ...)."""
    out = np.asarray(vecs[0], dtype=np.float64)
    for v in vecs[1:]:
        out = np.multiply.outer(out, np.asarray(v, dtype=np.float64))
    return out


def apply_axis(mat: np.ndarray, arr: np.ndarray, axis: int) -> np.ndarray:
    """Apply a square matrix along one axis of a C-ordered array (plain tensordot)."""
    moved = np.moveaxis(arr, axis, 0)
    res = np.tensordot(mat, moved, axes=([1], [0]))
    return np.moveaxis(res, 0, axis)


class ClosedFormBasis:
    """Diagonalisation by V = kron_a S_a with the closed-form eigenpairs.

    Modal ODE: c' = -lam c + ghat with ghat = Lambda_M^{-1} V^T F, where F is
    the consistent load vector and Lambda_M = kron_a diag(mu^M_a).
    Parity: pinned by the dense eigensolve route (``DenseBasis``), by
    V^T M V / V^T K V being diagonal, and by the paper's tables.
    """

    route = "closed_form"

    def __init__(self, n, box, D, periodic=()):
        self.n = tuple(int(v) for v in n)
        self.box = tuple(box)
        self.D = float(D)
        self.periodic = tuple(periodic) + (False,) * (len(self.n) - len(periodic))
        self.S = []
        self.muM_axes, self.muK_axes, self.h = [], [], []
        for a, na in enumerate(self.n):
            h, _ = axis_grid(box[a][0], box[a][1], na, self.periodic[a])
            if self.periodic[a]:
                muM, muK = axis_eigenvalues_periodic(na, h)
                self.S.append(dht_matrix(na))
            else:
                muM, muK = axis_eigenvalues(na, h)
                self.S.append(dst1_matrix(na))
            self.muM_axes.append(muM)
            self.muK_axes.append(muK)
            self.h.append(h)
        self.muM = outer_all(self.muM_axes)
        lam = np.zeros(self.n)
        for a in range(len(self.n)):
            shape = [1] * len(self.n)
            shape[a] = self.n[a]
            lam = lam + (self.muK_axes[a] / self.muM_axes[a]).reshape(shape)
        self.lam = self.D * lam

    def to_modal_from_load(self, F: np.ndarray) -> np.ndarray:
        """ghat = Lambda_M^{-1} V^T F (F nodal load, shape n)."""
        out = F
        for a, S in enumerate(self.S):
            out = apply_axis(S, out, a)
        return out / self.muM

    def to_nodal(self, c: np.ndarray) -> np.ndarray:
        """Nodal values u = V c."""
        out = c
        for a, S in enumerate(self.S):
            out = apply_axis(S, out, a)
        return out

    def to_modal_from_nodal(self, u: np.ndarray) -> np.ndarray:
        """c = V^T u for a nodal vector already in V_h (V orthogonal)."""
        return self.to_nodal(u)

    def norm2_weights(self) -> np.ndarray:
        """||v||_0^2 = sum_J muM_J c_J^2 for v = V c."""
        return self.muM

    def axis_modal_factor(self, a: int, F_axis: np.ndarray) -> np.ndarray:
        """1D factor (S_a F_a) / mu^M_a of a separable load (outer product of these)."""
        return (self.S[a] @ F_axis) / self.muM_axes[a]


class DenseBasis:
    """Diagonalisation by a dense generalized symmetric eigensolve of (K, M).

    Eigenvectors W are M-orthonormal (W^T M W = I, W^T K W = diag(lam)), so
    c = W^T M u, ghat = W^T F and u = W c.  Used on tiny grids only, as the
    independent route that pins ``ClosedFormBasis``.
    """

    route = "dense"

    def __init__(self, n, box, D, periodic=()):
        self.n = tuple(int(v) for v in n)
        M, K = assemble(self.n, box, D, periodic)
        self.M = M.toarray()
        self.K = K.toarray()
        lam, W = scipy.linalg.eigh(self.K, self.M)
        self.lam_flat = lam
        self.W = W
        self.lam = lam  # flat modal index

    def to_modal_from_load(self, F: np.ndarray) -> np.ndarray:
        return self.W.T @ F.reshape(-1)

    def to_nodal(self, c: np.ndarray) -> np.ndarray:
        return (self.W @ c).reshape(self.n)

    def to_modal_from_nodal(self, u: np.ndarray) -> np.ndarray:
        return self.W.T @ (self.M @ u.reshape(-1))

    def norm2_weights(self) -> np.ndarray:
        return np.ones_like(self.lam)
