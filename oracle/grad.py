"""Gradients with respect to the potential of H(V) = -1/2 Lap + diag(V), from
dense eigendecompositions (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

These are the textbook first-order perturbation formulas for a real
symmetric matrix with simple eigenvalues, written over the full spectrum
(numpy's eigh as one step), with no projection or iterative solve:

* eigenvalue: d lambda_c / d V_i = y_c(i)^2 (Hellmann-Feynman), so the
  gradient of sum_c w_c lambda_c is sum_c w_c y_c^2;
* eigenvector: d y_c / d V_i = sum_{j != c} y_j y_j(i) y_c(i) / (lambda_c -
  lambda_j), so for a loss L with G = dL/dY the gradient is
  dL/dV_i = sum_c y_c(i) b_c(i),  b_c = sum_{j != c} y_j (y_j^T g_c) /
  (lambda_c - lambda_j).

The GPU path splits b_c into the terms with j inside the computed block and a
shifted solve for the rest; the oracle keeps the single sum.
"""
from __future__ import annotations

import numpy as np


def eigval_grad(Y, w):
    """sum_c w_c Y[:, c]^2 for orthonormal eigenvectors Y (n x k)."""
    Y = np.asarray(Y, dtype=np.float64)
    return (Y ** 2) @ np.asarray(w, dtype=np.float64)


def eigvec_grad(H, idx, G):
    """dL/dV (n) for the eigenvectors idx of the dense symmetric H and
    G = dL/dY[:, idx] (n x len(idx)), with Y the eigenvectors numpy's eigh
    returns (G must be formed with those signs).  Returns (grad, lam, Y)."""
    lam, Y = np.linalg.eigh(np.asarray(H, dtype=np.float64))
    G = np.asarray(G, dtype=np.float64)
    grad = np.zeros(Y.shape[0])
    for col, c in enumerate(idx):
        coef = Y.T @ G[:, col]
        d = lam[c] - lam
        d[c] = np.inf                      # the j = c term is absent
        b = Y @ (coef / d)
        grad += Y[:, c] * b
    return grad, lam, Y
