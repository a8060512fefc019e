"""Closed-form gradient of a visibility loss, float64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The correction of Sec. 2.1 multiplies antenna i's spectra by
a_i[k] = g_i exp(-2 pi i k tau_i / K) before the cross-multiply, so every
emitted visibility is V_ij[k] = a_i[k] conj(a_j[k]) R_ij[k], where R is the
uncorrected visibility.  For the loss

    L = sum_{i<=j, k} |V_ij[k] - M_ij[k]|^2

(M a fixed model, by default the uncorrected instrument R, i.e. a = 1) the
Wirtinger derivative with respect to conj(a_m[k]) is, with E = V - M,

    dL/dconj(a_m) = sum_{j>=m} E_mj a_j conj(R_mj) + sum_{i<=m} conj(E_im) a_i R_im

and the returned gradients follow PyTorch's complex convention
(grad = dL/dRe + i dL/dIm = 2 dL/dconj):

    grad_g_m   = sum_k 2 dL/dconj(a_m[k]) * conj(exp(-2 pi i k tau_m / K))
    grad_tau_m = sum_k 2 Re( dL/dconj(a_m[k])^* * (-2 pi i k / K) * a_m[k] )
"""

import numpy as np

from .fx import baseline_pairs, correction_factors


def loss(R, gains, delays, K, M=None):
    """L = sum |a_i conj(a_j) R_ij - M_ij|^2 over emitted pairs and channels.

    ``R`` and ``M`` are ``[P][C]`` in ``baseline_pairs`` order.
    """
    R = np.asarray(R, np.complex128)
    N = len(gains)
    M = R if M is None else np.asarray(M, np.complex128)
    a = correction_factors(K, gains, delays, N=N)
    pairs = baseline_pairs(N)
    ii = np.array([p[0] for p in pairs])
    jj = np.array([p[1] for p in pairs])
    V = a[ii] * np.conj(a[jj]) * R
    return float(np.sum(np.abs(V - M) ** 2))


def loss_and_grad(R, gains, delays, K, M=None):
    """Return (L, grad_g[N] complex, grad_tau[N] real) for the loss above."""
    R = np.asarray(R, np.complex128)
    N = len(gains)
    C = R.shape[1]
    M = R if M is None else np.asarray(M, np.complex128)
    a = correction_factors(K, gains, delays, N=N)
    pairs = baseline_pairs(N)
    E = np.empty_like(R)
    for p, (i, j) in enumerate(pairs):
        E[p] = a[i] * np.conj(a[j]) * R[p] - M[p]
    L = float(np.sum(np.abs(E) ** 2))

    dconj = np.zeros((N, C), np.complex128)        # dL/dconj(a_m[k])
    for p, (i, j) in enumerate(pairs):
        # E_ij depends on conj(a_j); conj(E_ij) depends on conj(a_i).
        dconj[j] += np.conj(E[p]) * a[i] * R[p]
        dconj[i] += E[p] * a[j] * np.conj(R[p])

    grad_a = 2.0 * dconj
    tau = np.asarray(delays, np.float64)
    k = np.arange(C, dtype=np.float64)
    phi = np.exp(-2j * np.pi * np.outer(tau, k) / K)
    grad_g = np.sum(grad_a * np.conj(phi), axis=1)
    da_dtau = (-2j * np.pi * k[None, :] / K) * a
    grad_tau = np.sum(np.real(np.conj(grad_a) * da_dtau), axis=1)
    return L, grad_g, grad_tau
