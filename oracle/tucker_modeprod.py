"""FP64 Tucker block-MM sweep and objective through successive mode-n products (test
infrastructure only, like the rest of this package).

The C oracle (``ntf_oracle.c``) rebuilds every entry of Xhat from the full core (prod_n J_n
products per entry), which is exact but far too slow for a 400 x 400 x 400 tensor with a
32 x 32 x 32 core.  This module computes the same quantities in FP64 with plain PyTorch CPU
ops, using the mode-n product of Section 3.3 ("mode-n product": (T x_n M)_{..i_n..} =
sum_{j_n} T_{..j_n..} M_{i_n j_n}) as its only contraction primitive:

  * Xhat = G x_1 A^(1) x_2 A^(2) ... x_N A^(N)                (Section 3.3, Tucker model)
  * P = X (.) max(Xhat, eps)^(beta - 2), Q = max(Xhat, eps)^(beta - 1)   (Section 4.1;
    X floored at eps_x only at beta = 0, the reading of Remark "The case beta = 0")
  * core: P_core = P x_1 A^(1)T ... x_N A^(N)T, Q_core likewise, then
    G <- max(G (.) (P_core / Q_core)^gamma(beta), eps)         (Appendix C, eq. (block_core_num_den);
    Theorem "Tucker block multiplicative updates")
  * factor n: Num^(n)_{i_n j_n} = sum_{i_-n} P_i B^(n)_{j_n, i_-n} with the partial tensor
    B^(n) = G x_{m != n} A^(m) (eq. (block_Bn)); evaluated as
    sum_{j_-n} (P x_{m != n} A^(m)T)_{..i_n..} G_{..j_n..} -- the same sum over i_-n and j_-n
    with the order of the two finite sums exchanged (eqs. (block_factor_num/den))
  * blocks in the order core, then modes 1..N, each from the current blocks (Appendix C.2).

Pinned in ``tests/test_oracle_pins.py`` against ``ntfo_tucker_mu_sweep`` and
``ntfo_tucker_objective`` of the C oracle.
"""
import numpy as np


def _torch():
    import torch
    return torch


def mode_product(T, M, n):
    """T x_n M: contracts mode n of T (size J) with the columns of M (I x J)."""
    torch = _torch()
    out = torch.tensordot(T, M, dims=([n], [1]))  # the new mode is last
    return torch.movedim(out, -1, n)


def tucker_full(G, A):
    """Xhat = G x_1 A^(1) ... x_N A^(N) in FP64 (torch CPU tensors or numpy arrays)."""
    torch = _torch()
    T = torch.as_tensor(np.asarray(G, dtype=np.float64))
    for n, a in enumerate(A):
        T = mode_product(T, torch.as_tensor(np.asarray(a, dtype=np.float64)), n)
    return T


def _floor_x(X, beta, eps_x):
    torch = _torch()
    return torch.clamp(X, min=eps_x) if beta == 0.0 else X


def dbeta_sum(X, Xh, beta, eps=1e-12, eps_x=1e-12):
    """sum_i d_beta(X_i | max(Xhat_i, eps)) (Section 3.2, Definition "beta-divergence")."""
    torch = _torch()
    y = torch.clamp(Xh, min=eps)
    x = _floor_x(X, beta, eps_x)
    if beta == 1.0:
        pos = x > 0
        xl = torch.where(pos, x * torch.log(torch.where(pos, x, torch.ones_like(x)) / y), torch.zeros_like(x))
        return float((xl - x + y).sum())
    if beta == 0.0:
        u = x / y
        return float((u - torch.log(u) - 1.0).sum())
    d = (x ** beta + (beta - 1.0) * y ** beta - beta * x * y ** (beta - 1.0)) / (beta * (beta - 1.0))
    return float(d.sum())


def tucker_objective(X, G, A, beta, eps=1e-12, eps_x=1e-12):
    torch = _torch()
    Xt = torch.as_tensor(np.asarray(X, dtype=np.float64)) if not torch.is_tensor(X) else X.double()
    return dbeta_sum(Xt, tucker_full(G, A), beta, eps, eps_x)


def _gamma(beta):
    # Remark "Exponent gamma(beta)": 1 / (2 - beta) for beta < 1, else 1
    return 1.0 / (2.0 - beta) if beta < 1.0 else 1.0


def _mu(pre, num, den, beta, eps):
    torch = _torch()
    return torch.clamp(pre * (num / den) ** _gamma(beta), min=eps)


def tucker_mu_sweep(X, G, A, beta, eps=1e-12, eps_x=1e-12):
    """One Tucker block-MM sweep (core, then modes 1..N).  Returns (G, [A], F_in) as numpy
    FP64 arrays; F_in is the objective of the incoming iterate."""
    torch = _torch()
    Xt = torch.as_tensor(np.asarray(X, dtype=np.float64)) if not torch.is_tensor(X) else X.double()
    Gt = torch.as_tensor(np.array(G, dtype=np.float64))
    At = [torch.as_tensor(np.array(a, dtype=np.float64)) for a in A]
    N = len(At)
    x = _floor_x(Xt, beta, eps_x)

    def powers():
        y = torch.clamp(tucker_full(Gt, At), min=eps)
        return x * y ** (beta - 2.0), y ** (beta - 1.0), y

    P, Q, y = powers()
    F_in = dbeta_sum(Xt, y, beta, eps, eps_x)
    # core block
    Pc, Qc = P, Q
    for n in range(N):
        Pc = mode_product(Pc, At[n].T, n)
        Qc = mode_product(Qc, At[n].T, n)
    Gt = _mu(Gt, Pc, Qc, beta, eps)
    # factor blocks
    for n in range(N):
        P, Q, _ = powers()
        Pn, Qn = P, Q
        for m in range(N):
            if m != n:
                Pn = mode_product(Pn, At[m].T, m)
                Qn = mode_product(Qn, At[m].T, m)
        others = [m for m in range(N) if m != n]
        num = torch.tensordot(Pn, Gt, dims=(others, others))  # I_n x J_n
        den = torch.tensordot(Qn, Gt, dims=(others, others))
        At[n] = _mu(At[n], num, den, beta, eps)
    return Gt.numpy(), [a.numpy() for a in At], F_in
