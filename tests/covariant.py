"""Independent 4-D (covariant) statements used to pin the oracle's 3+1 formulas.

Everything here is built from the definitions in Sec. 2 of the paper, not from
the Valencia closed forms: the 4-metric from the ADM split (Eq. 5), the
stress-energy tensor (Eq. 2), the dual Faraday tensor (Eq. 3) with b^mu fixed by
b.u = 0 and the Eulerian field B^i = n_mu (*F)^{mu i}, and the projections onto
the normal observer n_mu = (-alpha, 0, 0, 0).  Conserved densities, fluxes and
sources then follow from writing the covariant laws of Eq. 1 in conservation
form (1/sqrt(-g)) d_mu (sqrt(-g) V^mu), with no use of Eqs. 6-9.
"""
import numpy as np


def four_metric(alpha, beta, g6):
    g = np.array([[g6[0], g6[1], g6[2]], [g6[1], g6[3], g6[4]], [g6[2], g6[4], g6[5]]], dtype=float)
    beta = np.asarray(beta, float)
    bl = g @ beta
    G = np.zeros((4, 4))
    G[0, 0] = -alpha * alpha + beta @ bl
    G[0, 1:] = bl
    G[1:, 0] = bl
    G[1:, 1:] = g
    return G, g


def fluid(alpha, beta, g6, rho, w, P, Bd, gamma_ad):
    """Covariant quantities of one state.  w^i = W v^i, Bd = densitised B~^i."""
    G, g = four_metric(alpha, beta, g6)
    Gi = np.linalg.inv(G)
    sdet = np.sqrt(np.linalg.det(g))
    B = np.asarray(Bd, float) / sdet
    w = np.asarray(w, float)
    W = np.sqrt(1.0 + w @ g @ w)
    v = w / W
    beta = np.asarray(beta, float)
    u = np.zeros(4)
    u[0] = W / alpha
    u[1:] = W * (v - beta / alpha)
    n_lo = np.array([-alpha, 0.0, 0.0, 0.0])
    # b^mu from b.u = 0 and B^i = n_mu (b^mu u^i - b^i u^mu) = -alpha (b^0 u^i - b^i u^0)
    A = np.zeros((4, 4))
    rhs = np.zeros(4)
    A[0, :] = G @ u            # b_mu u^mu = 0
    for i in range(3):
        A[1 + i, 0] = -alpha * u[1 + i]
        A[1 + i, 1 + i] = alpha * u[0]
        rhs[1 + i] = B[i]
    bvec = np.linalg.solve(A, rhs)
    b2 = bvec @ G @ bvec
    eps = P / ((gamma_ad - 1.0) * rho)
    h = 1.0 + eps + P / rho
    T = (rho * h + b2) * np.outer(u, u) + (P + 0.5 * b2) * Gi - np.outer(bvec, bvec)
    Fd = np.outer(bvec, u) - np.outer(u, bvec)   # (*F)^{mu nu}
    return dict(G=G, Gi=Gi, g=g, sdet=sdet, u=u, b=bvec, b2=b2, T=T, Fd=Fd, n_lo=n_lo, W=W, v=v, B=B,
                rho=rho, alpha=alpha, beta=beta, h=h)


def conserved(f):
    """Densitised D~, S~_i, tau~ as projections of rho u and T onto n."""
    T, G, alpha, sdet = f["T"], f["G"], f["alpha"], f["sdet"]
    D = -f["n_lo"] @ f["u"] * f["rho"]                      # rho W
    T_mix = T @ G                                             # T^mu_nu
    S = np.array([-(f["n_lo"] @ T_mix[:, 1 + i]) for i in range(3)])   # -n_mu T^mu_i
    E = f["n_lo"] @ T @ f["n_lo"]                             # n_mu n_nu T^{mu nu}
    return sdet * np.array([D, S[0], S[1], S[2], E - D])


def fluxes(f, d):
    """Densitised fluxes along direction d: sqrt(-g) V^d of the conserved currents,
    and of the induction law (Eq. 4c) for the two transverse B components."""
    T, G, alpha, sdet = f["T"], f["G"], f["alpha"], f["sdet"]
    sg = alpha * sdet
    j = 1 + d
    FD = sg * f["rho"] * f["u"][j]
    T_mix = T @ G
    FS = [sg * T_mix[j, 1 + i] for i in range(3)]
    # energy current: -n_nu T^{mu nu} - rho u^mu  (E - D)
    Fe = sg * (-(T[j, :] @ f["n_lo"])) - FD
    t1, t2 = (d + 1) % 3, (d + 2) % 3
    FB1 = sg * f["Fd"][1 + t1, j]
    FB2 = sg * f["Fd"][1 + t2, j]
    return np.array([FD, FS[0], FS[1], FS[2], Fe, FB1, FB2])


def speeds_flat_hydro(v, cs):
    """Characteristic speeds along a flow v in flat space (relativistic velocity addition)."""
    return (v - cs) / (1 - v * cs), (v + cs) / (1 + v * cs)
