"""Exact laws of the shaken dynamics on tiny tori, by full enumeration.

TEST INFRASTRUCTURE ONLY.  Written from the paper's definitions (Section 2):

* neighbours x^up=(i,j+1), x^right=(i+1,j), x^down=(i,j-1), x^left=(i-1,j) on
  the torus (Z/LZ)^2, linear index u = j*L + i;
* fields (Eq. "urdl"): <-h_x(sigma) = J(sigma_{x down} + sigma_{x left}) + q sigma_x,
  ->h_x(tau) = J(tau_{x up} + tau_{x right}) + q tau_x;
* half-step kernels (Eqs. "leftTrans", "rightTrans"): products over sites of
  e^{zeta h} / (2 cosh h);
* shaken kernel P^sq(sigma, sigma') = sum_tau P_A(sigma, tau) P_B(tau, sigma')
  (the sigma-marginal of the alternate chain);
* its closed-form stationary law pi_s(sigma) = Z_sigma / Z with
  Z_sigma = sum_eta e^{-H(sigma, eta)} = prod_u 2 cosh(<-h_u(sigma));
* the pair Gibbs measure pi_2(sigma, tau) proportional to e^{-H(sigma, tau)}
  (Eq. "gs_ham2");
* the critical curve J_c(q) = atanh(sqrt(tanh^2 q + 1) - tanh q) (Eq. "J_di_q").

States are integer codes: bit u of the code set iff the spin at u is +1.
"""
from __future__ import annotations

import numpy as np


def neighbours(L: int):
    """Linear indices of x^up, x^right, x^down, x^left for every site x."""
    j, i = np.divmod(np.arange(L * L), L)
    up = ((j + 1) % L) * L + i
    right = j * L + (i + 1) % L
    down = ((j - 1) % L) * L + i
    left = j * L + (i - 1) % L
    return up, right, down, left


def spin_table(N: int) -> np.ndarray:
    """S[code, u] = +1 if bit u of code is set, else -1; shape (2^N, N)."""
    codes = np.arange(2 ** N, dtype=np.int64)
    bits = (codes[:, None] >> np.arange(N)[None, :]) & 1
    return (2 * bits - 1).astype(np.int64)


def left_fields(S: np.ndarray, L: int, q: float, J: float) -> np.ndarray:
    _, _, down, left = neighbours(L)
    return J * (S[:, down] + S[:, left]) + q * S


def right_fields(S: np.ndarray, L: int, q: float, J: float) -> np.ndarray:
    up, right, _, _ = neighbours(L)
    return J * (S[:, up] + S[:, right]) + q * S


def field_classes(S: np.ndarray, L: int, which: str) -> np.ndarray:
    """Threshold-table index k = 3*[s=+1] + n (n = number of +1 neighbours in
    the field) for every state and site."""
    up, right, down, left = neighbours(L)
    a, b = (down, left) if which == "left" else (up, right)
    n = (S[:, a] > 0).astype(np.int64) + (S[:, b] > 0).astype(np.int64)
    return 3 * (S > 0).astype(np.int64) + n


def _kernel_from_pup(p_up: np.ndarray, S: np.ndarray) -> np.ndarray:
    """K[a, b] = prod_u P(spin_u of state b | p_up[a, u])."""
    up_mask = S[None, :, :] > 0
    fac = np.where(up_mask, p_up[:, None, :], 1.0 - p_up[:, None, :])
    return np.prod(fac, axis=2)


def half_step_kernels(L: int, q: float, J: float, T: np.ndarray | None = None):
    """(P_A, P_B) as dense matrices over state codes.  With T=None the exact
    probabilities e^{h}/(2 cosh h) are used; with a 6-entry threshold table the
    quantised probabilities T[k] / 2^32 are used instead."""
    S = spin_table(L * L)
    if T is None:
        pA = 0.5 * (1.0 + np.tanh(left_fields(S, L, q, J)))
        pB = 0.5 * (1.0 + np.tanh(right_fields(S, L, q, J)))
    else:
        tab = np.asarray(T, dtype=np.float64) / 2.0 ** 32
        pA = tab[field_classes(S, L, "left")]
        pB = tab[field_classes(S, L, "right")]
    return _kernel_from_pup(pA, S), _kernel_from_pup(pB, S)


def shaken_kernel(L: int, q: float, J: float, T: np.ndarray | None = None) -> np.ndarray:
    PA, PB = half_step_kernels(L, q, J, T)
    return PA @ PB


def stationary(P: np.ndarray) -> np.ndarray:
    """Stationary row vector of a stochastic matrix (direct linear solve)."""
    n = P.shape[0]
    A = P.T - np.eye(n)
    A[-1, :] = 1.0
    b = np.zeros(n)
    b[-1] = 1.0
    pi = np.linalg.solve(A, b)
    return pi / pi.sum()


def pi_s_closed_form(L: int, q: float, J: float) -> np.ndarray:
    """pi_s(sigma) proportional to prod_u 2 cosh(<-h_u(sigma))."""
    S = spin_table(L * L)
    h = left_fields(S, L, q, J)
    logw = np.sum(np.log(2.0 * np.cosh(h)), axis=1)
    w = np.exp(logw - logw.max())
    return w / w.sum()


def pair_hamiltonian(L: int, q: float, J: float) -> np.ndarray:
    """H[sigma_code, tau_code] = -sum_x [J sigma_x (tau_{x up} + tau_{x right})
    + q sigma_x tau_x]."""
    S = spin_table(L * L)
    up, right, _, _ = neighbours(L)
    coupling = S[:, None, :] * (J * (S[None, :, up] + S[None, :, right]) + q * S[None, :, :])
    return -np.sum(coupling, axis=2)


def pi_2(L: int, q: float, J: float) -> np.ndarray:
    H = pair_hamiltonian(L, q, J)
    w = np.exp(-(H - H.min()))
    return w / w.sum()


def critical_J(q):
    """J_c(q) of Eq. J_di_q (the solution of 1 = 2 tanh J tanh q + tanh^2 J)."""
    t = np.tanh(q)
    return np.arctanh(np.sqrt(t * t + 1.0) - t)


# ---- square-lattice Ising model and its checkerboard heat bath (Section 3.2)

def square_energy(L: int, J: float) -> np.ndarray:
    """H_G(s) = -J sum_x s_x (s_{x up} + s_{x right}) for every state code."""
    S = spin_table(L * L)
    up, right, _, _ = neighbours(L)
    return -J * np.sum(S * (S[:, up] + S[:, right]), axis=1)


def square_gibbs(L: int, J: float) -> np.ndarray:
    H = square_energy(L, J)
    w = np.exp(-(H - H.min()))
    return w / w.sum()


def checkerboard_kernel(L: int, J: float, parity: int, T5=None) -> np.ndarray:
    """Heat-bath redraw of the sites with (i + j) % 2 == parity given the
    others, as a dense matrix over state codes (exact probabilities
    e^{h}/(2 cosh h), h = J * sum of the four neighbours, or the quantised
    T5[n] / 2^32 with n the number of + neighbours)."""
    N = L * L
    S = spin_table(N)
    up, right, down, left = neighbours(L)
    j, i = np.divmod(np.arange(N), L)
    active = ((i + j) % 2) == parity
    nplus = (S[:, up] > 0).astype(np.int64) + (S[:, down] > 0) + (S[:, left] > 0) + (S[:, right] > 0)
    if T5 is None:
        p_up = 0.5 * (1.0 + np.tanh(J * (2.0 * nplus - 4.0)))
    else:
        p_up = np.asarray(T5, dtype=np.float64)[nplus] / 2.0 ** 32
    n_states = 2 ** N
    K = np.zeros((n_states, n_states))
    act = np.nonzero(active)[0]
    for a in range(n_states):
        base = S[a].copy()
        for bits in range(2 ** len(act)):
            prob = 1.0
            new = base.copy()
            for k, site in enumerate(act):
                v = 1 if (bits >> k) & 1 else -1
                new[site] = v
                prob *= p_up[a, site] if v > 0 else 1.0 - p_up[a, site]
            code = int(np.sum((new > 0).astype(np.int64) << np.arange(N)))
            K[a, code] += prob
    return K
