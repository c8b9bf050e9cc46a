"""Plain NumPy Davidson eigensolver (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 3.3 of the paper lists the steps of the CI eigensolver: (1) build and
diagonalise an initial subspace matrix, which needs an initial sigma vector;
(2) compute the preconditioner; (3) multiply the residual by the inverse
(diagonal) Hessian and orthogonalise it against all previous vectors; (4) form
the new sigma vector and diagonalise the enlarged projected matrix; return to
(2) until converged.  The paper calls LUCIA's variant "modified
inverted-Davidson" without defining it, so this oracle takes these readings:

* block Davidson-Liu (Davidson 1975) with the diagonal preconditioner
  ``t_k = -(H_diag - E_k)^{-1} r_k``, ``r_k = H x_k - E_k x_k``;
* a denominator with ``|H_II - E| < 1e-8`` is replaced by ``+-1e-8`` (its sign
  kept; zero counts as positive);
* step (3)'s "diagonalization to all previous vectors" is read as
  orthogonalisation: classical Gram-Schmidt applied twice, then normalisation;
  a correction whose norm falls below 1e-10 is dropped;
* converged when, for every root, ``|E_k - E_k(previous)| < tol`` and
  ``||r_k|| < sqrt(tol)``;
* initial guess: unit vectors on the ``nroots`` smallest diagonal elements,
  ties broken by the lower determinant index;
* when the subspace would exceed ``max_subspace`` it collapses to the current
  Ritz vectors (and their sigma vectors).
"""
from __future__ import annotations

import numpy as np


def initial_guess(diag: np.ndarray, nroots: int) -> np.ndarray:
    order = np.argsort(diag, kind="stable")[:nroots]
    X = np.zeros((nroots, diag.size))
    X[np.arange(nroots), order] = 1.0
    return X


def precondition(r: np.ndarray, diag: np.ndarray, e: float, floor: float = 1e-8) -> np.ndarray:
    d = diag - e
    small = np.abs(d) < floor
    d = np.where(small, np.where(d < 0, -floor, floor), d)
    return -r / d


def davidson(matvec, diag, nroots=1, tol=1e-10, max_subspace=24, max_iter=200, guess=None):
    """Lowest ``nroots`` eigenpairs of a real symmetric operator.

    Returns dict(energies, vectors [nroots, N], converged, iterations,
    history=[(energies, residual_norms), ...]).
    """
    diag = np.asarray(diag, dtype=np.float64)
    N = diag.size
    nroots = min(nroots, N)
    max_subspace = max(max_subspace, 2 * nroots)
    B = initial_guess(diag, nroots) if guess is None else np.array(guess, dtype=np.float64).reshape(-1, N)
    # orthonormalise the starting block
    Q, _ = np.linalg.qr(B.T)
    B = Q.T.copy()
    S = np.array([matvec(b) for b in B])
    e_prev = np.full(nroots, np.inf)
    history = []
    converged = False
    it = 0
    for it in range(1, max_iter + 1):
        A = B @ S.T
        A = 0.5 * (A + A.T)
        w, v = np.linalg.eigh(A)
        w, v = w[:nroots], v[:, :nroots]
        X = v.T @ B
        HX = v.T @ S
        R = HX - w[:, None] * X
        rn = np.linalg.norm(R, axis=1)
        history.append((w.copy(), rn.copy()))
        if np.all(np.abs(w - e_prev) < tol) and np.all(rn < np.sqrt(tol)):
            converged = True
            break
        e_prev = w.copy()
        if B.shape[0] + nroots > max_subspace:
            B, S = X.copy(), HX.copy()
        new = []
        for k in range(nroots):
            t = precondition(R[k], diag, w[k])
            for _ in range(2):
                t = t - B.T @ (B @ t)
                for q in new:
                    t = t - q * (q @ t)
            nt = np.linalg.norm(t)
            if nt < 1e-10:
                continue
            new.append(t / nt)
        if not new:
            # nothing left to add: residuals below the floor of the method
            converged = bool(np.all(rn < np.sqrt(tol)))
            break
        Snew = np.array([matvec(t) for t in new])
        B = np.vstack([B, np.array(new)])
        S = np.vstack([S, Snew])
    return {
        "energies": w,
        "vectors": X,
        "converged": converged,
        "iterations": it,
        "history": history,
    }
