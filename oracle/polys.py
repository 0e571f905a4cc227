"""One-dimensional polynomial tools (oracle, test infrastructure only).

Gauss-Legendre points for the solution and flux points (Section 3.1: points
"distributed according to the Gauss-Legendre points"), Legendre and Jacobi
polynomials for the orthonormal modal bases Psi of the Vandermonde matrix,
Lagrange interpolation (the nodal basis l_i) and the left Radau polynomial used
as the DG-recovering correction function g (Section 3.1, Step 3).
"""
import math

import numpy as np


def gauss_legendre(n):
    """n-point Gauss-Legendre rule on [-1, 1] by Golub-Welsch.

    The nodes are the eigenvalues of the symmetric Jacobi matrix of the
    Legendre recurrence (off-diagonal k / sqrt(4k^2 - 1)); the weights are
    2 v_0^2 with v the normalised eigenvectors.
    """
    if n == 1:
        return np.zeros(1), np.full(1, 2.0)
    k = np.arange(1, n, dtype=np.float64)
    off = k / np.sqrt(4.0 * k * k - 1.0)
    Jm = np.diag(off, 1) + np.diag(off, -1)
    x, v = np.linalg.eigh(Jm)
    w = 2.0 * v[0, :] ** 2
    # symmetrise to remove round-off asymmetry
    x = 0.5 * (x - x[::-1])
    w = 0.5 * (w + w[::-1])
    return x, w


def jacobi(n, a, b, x):
    """Jacobi polynomial P_n^{(a,b)}(x) by the three-term recurrence."""
    x = np.asarray(x, dtype=np.float64)
    p0 = np.ones_like(x)
    if n == 0:
        return p0
    p1 = 0.5 * (a - b + (a + b + 2.0) * x)
    for k in range(2, n + 1):
        c1 = 2.0 * k * (k + a + b) * (2.0 * k + a + b - 2.0)
        c2 = (2.0 * k + a + b - 1.0) * (a * a - b * b)
        c3 = (2.0 * k + a + b - 2.0) * (2.0 * k + a + b - 1.0) * (2.0 * k + a + b)
        c4 = 2.0 * (k + a - 1.0) * (k + b - 1.0) * (2.0 * k + a + b)
        p0, p1 = p1, ((c2 + c3 * x) * p1 - c4 * p0) / c1
    return p1


def jacobi_deriv(n, a, b, x):
    """d/dx P_n^{(a,b)} = (n + a + b + 1)/2 * P_{n-1}^{(a+1,b+1)}."""
    if n == 0:
        return np.zeros_like(np.asarray(x, dtype=np.float64))
    return 0.5 * (n + a + b + 1.0) * jacobi(n - 1, a + 1.0, b + 1.0, x)


def jacobi_norm(n, a, b):
    """Squared L2 norm of P_n^{(a,b)} with weight (1-x)^a (1+x)^b on [-1,1]."""
    return (2.0 ** (a + b + 1.0) / (2.0 * n + a + b + 1.0)
            * math.gamma(n + a + 1.0) * math.gamma(n + b + 1.0)
            / (math.gamma(n + a + b + 1.0) * math.gamma(n + 1.0)))


def legendre(n, x):
    return jacobi(n, 0.0, 0.0, x)


def legendre_deriv(n, x):
    return jacobi_deriv(n, 0.0, 0.0, x)


def lagrange_matrix(nodes, x, deriv=False):
    """Matrix B[k, j] = l_j(x_k) (or l_j'(x_k)) for the Lagrange basis on `nodes`.

    Direct product formula l_j(x) = prod_{m != j} (x - x_m) / (x_j - x_m) and
    its derivative by the product rule.
    """
    nodes = np.asarray(nodes, dtype=np.float64)
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    n = nodes.size
    B = np.zeros((x.size, n))
    for j in range(n):
        den = np.prod([nodes[j] - nodes[m] for m in range(n) if m != j])
        if not deriv:
            num = np.ones_like(x)
            for m in range(n):
                if m != j:
                    num = num * (x - nodes[m])
            B[:, j] = num / den
        else:
            tot = np.zeros_like(x)
            for r in range(n):
                if r == j:
                    continue
                term = np.ones_like(x)
                for m in range(n):
                    if m != j and m != r:
                        term = term * (x - nodes[m])
                tot = tot + term
            B[:, j] = tot / den
    return B


def radau_left(p, x):
    """Left correction function g_L = R_{R,p+1} = (-1)^{p+1}/2 (P_{p+1} - P_p):
    g_L(-1) = 1, g_L(1) = 0, degree p+1 (Huynh's DG-recovering choice)."""
    return (-1.0) ** (p + 1) * 0.5 * (legendre(p + 1, x) - legendre(p, x))


def radau_left_deriv(p, x):
    return (-1.0) ** (p + 1) * 0.5 * (legendre_deriv(p + 1, x) - legendre_deriv(p, x))
