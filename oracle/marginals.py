"""Adiabatic-basis wavepacket marginals of Sec. III ("Wavepacket dynamics") in plain numpy FP64.

Test infrastructure only: imported by tests/ and never by the library or its binding.

The paper plots P^(ad)_jk(q; t) = integral dp W^(ad)_jk(p, q; t), the Wigner distribution of the zeroth
hierarchy tier taken to the adiabatic basis and integrated over p.  The p-integral of a Wigner
distribution is the density matrix on its diagonal, rho_jk(q, q), and the adiabatic basis change
rho^(ad)(q, q') = V(q)^T rho(q, q') V(q') is local in q on that diagonal, so
    P^(ad)(q) = V(q)^T [dp sum_l W^(0)(q, p_l)] V(q)
exactly.  V(q) holds the eigenvectors of the real symmetric diabatic matrix U_jk(q), ascending
eigenvalue first, each signed so that its first component of largest magnitude (within 1e-9) is
positive.
"""
import numpy as np


def diabatic_matrix(U_table):
    """U_jk(q_i) from the potential table [S][S][nq][np + 1] (column np/2 is the zero offset):
    returns [nq][S][S]."""
    n_t = U_table.shape[-1]
    return np.ascontiguousarray(np.moveaxis(U_table[:, :, :, (n_t - 1) // 2], -1, 0))


def adiabatic_basis(Uq):
    """Eigenvectors of each U(q_i): v[i][j][a] = component j of adiabatic state a (numpy eigh, ascending),
    with the sign convention above."""
    nq, S, _ = Uq.shape
    V = np.empty_like(Uq)
    for i in range(nq):
        w, v = np.linalg.eigh(0.5 * (Uq[i] + Uq[i].T))
        for a in range(S):
            col = v[:, a]
            mx = np.abs(col).max()
            lead = int(np.nonzero(np.abs(col) >= mx - 1e-9)[0][0])
            V[i, :, a] = -col if col[lead] < 0 else col
    return V


def coordinate_marginals(W0, dp):
    """rho_jk(q_i) = dp sum_l W^(0)_jk(q_i, p_l) for the zeroth tier W0 [S][S][nq][np]."""
    return W0.sum(axis=-1) * dp


def adiabatic_marginals(W, U_table, dp):
    """P^(ad)_ab(q_i) for a state W [n_elem][S][S][nq][np] (zeroth tier first): [S][S][nq] complex."""
    rho = coordinate_marginals(W[0], dp)
    V = adiabatic_basis(diabatic_matrix(U_table))
    return np.einsum("ija,jki,ikb->abi", V, rho, V)
