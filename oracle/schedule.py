"""The paper's stepwise coupling schedule and its Trotter-error estimates.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2.2: the coupling of the m-th substep of the k-th step is
g_{k,m} = (k-1) g_s + m delta, delta = g_s / n (right end of each substep);
Eq. (error1)/(asymtotal) and Eq. (symmerror)/(total) estimate the total error.
"""

from __future__ import annotations


def g_values(N_s, n, g_s):
    delta = g_s / n
    return [(k - 1) * g_s + m * delta for k in range(1, N_s + 1) for m in range(1, n + 1)]


def sum_g_closed(N_s, n, g_s):
    """Closed form of sum_{k,m} g_{k,m} printed in Sec. 2.2."""
    return 0.5 * (N_s * N_s * n + N_s) * g_s


def sum_g2_closed(N_s, n, g_s):
    """Closed form of sum_{k,m} g_{k,m}^2 printed in Sec. 2.2."""
    return ((N_s - 1) * N_s * (2 * N_s - 1) * n * g_s ** 2 / 6
            + N_s * n * (n + 1) * (2 * n + 1) * g_s ** 2 / (6 * n * n)
            + N_s * (N_s - 1) * (n + 1) * g_s ** 2 / 2)


def delta_asym_total(N_s, N_p, g_s, t_s, n):
    """Eq. (asymtotal), leading term."""
    return N_s ** 2 * N_p * g_s * t_s ** 2 / n


def delta_sym_total(N_s, N_p, g_s, t_s, n):
    """Eq. (total), leading term."""
    return 4.0 / 9.0 * N_s ** 3 * N_p * g_s ** 2 * t_s ** 3 / n ** 2
