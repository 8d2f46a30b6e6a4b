"""Linear stability analysis of the settling interface (Sec. 3), in lattice units:
``growth_rate`` with one transported scalar (no density-altering scalar: S* = 0) and
``growth_rate_sugar`` with the sugar scalar S as well (the paper's full K/W problem).

TEST INFRASTRUCTURE ONLY (reference for the coupled early-time growth rate).

Model (Sec. 3.1-3.2 with the sugar row and column removed): 2D, x periodic, y
vertical between no-slip walls at y = 0 and y = H; stream function psi with
u = (d psi/dy, -d psi/dx), vorticity omega = -lap psi; base state at rest with
concentration profile cbar(y) (an erf profile, Eqs. phi_bs); buoyancy force
F = -A c e_y.  Normal modes exp(i k x + sigma t) of
    d omega/dt = nu lap omega - A dc/dx
    d c/dt + v dcbar/dy - Vs dc/dy = kappa lap c
give the generalised eigenproblem K x = sigma W x for x = (psi, c), with
M = D^2 - k^2:
    sigma M psi = nu M^2 psi + i k A c
    sigma c     = i k cbar' psi + (Vs D + kappa M) c
(the paper's K and W of Sec. 3.2 with the S rows dropped; omega eliminated).
Discretised with second-order finite differences on a uniform grid with points on
the walls: psi = psi' = 0 (clamped, no-slip), dc/dy = 0 (Neumann, Eq. neum1).
"""
import numpy as np
from scipy import linalg
from scipy.special import erf


def erf_profile(y, yc, delta, lower=0.0, upper=1.0):
    """cbar(y) = lower + (upper - lower) (1 + erf((y - yc)/delta)) / 2 (Eq. phi_bs form)."""
    return lower + (upper - lower) * 0.5 * (1.0 + erf((y - yc) / delta))


def fit_erf(y, c):
    """Least-squares fit of erf_profile to a measured mean profile; returns (yc, delta)."""
    from scipy.optimize import curve_fit
    i = int(np.argmin(np.abs(c - 0.5 * (c.min() + c.max()))))
    p0 = (y[i], 2.0)
    (yc, delta), _ = curve_fit(lambda yy, a, b: erf_profile(yy, a, b, c.min(), c.max()), y, c, p0=p0)
    return yc, abs(delta)


def growth_rate(k, H, nu, A, kappa, vs, cbar_fn, m=400):
    """Largest real part of sigma(k) for the interface problem on (0, H) with m intervals."""
    h = H / m
    y = np.linspace(0.0, H, m + 1)
    n = m - 1                      # interior psi unknowns (psi = 0 on the walls)
    yi = y[1:-1]
    # psi operators on interior points; clamped walls: psi_0 = 0, ghost psi_{-1} = psi_1
    D2 = (np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)) / h**2
    D4 = (np.diag(6.0 * np.ones(n)) + np.diag(-4.0 * np.ones(n - 1), 1) + np.diag(-4.0 * np.ones(n - 1), -1)
          + np.diag(np.ones(n - 2), 2) + np.diag(np.ones(n - 2), -2))
    D4[0, 0] += 1.0                # ghost psi_{-1} = psi_1 enters row 1 through the +1 coefficient
    D4[-1, -1] += 1.0
    D4 /= h**4
    I = np.eye(n)
    Mpsi = D2 - k**2 * I
    M2psi = D4 - 2.0 * k**2 * D2 + k**4 * I
    # c on all m+1 points with Neumann walls (ghost c_{-1} = c_1)
    nc = m + 1
    Dc = np.zeros((nc, nc))
    D2c = np.zeros((nc, nc))
    for j in range(nc):
        jm, jp = j - 1, j + 1
        if jm < 0:
            jm = 1
        if jp > m:
            jp = m - 1
        if 0 < j < m:
            Dc[j, jp] += 0.5 / h
            Dc[j, jm] -= 0.5 / h
        D2c[j, jp] += 1.0 / h**2
        D2c[j, jm] += 1.0 / h**2
        D2c[j, j] -= 2.0 / h**2
    Mc = D2c - k**2 * np.eye(nc)
    cb = cbar_fn(y)
    dcb = np.gradient(cb, y)
    # couplings: c (all points) -> psi rows (interior), psi (interior) -> c rows (interior)
    Cpc = np.zeros((n, nc), dtype=complex)
    Cpc[:, 1:-1] = 1j * k * A * np.eye(n)
    Ccp = np.zeros((nc, n), dtype=complex)
    Ccp[1:-1, :] = 1j * k * np.diag(dcb[1:-1])
    K = np.block([[nu * M2psi.astype(complex), Cpc], [Ccp, (vs * Dc + kappa * Mc).astype(complex)]])
    W = np.block([[Mpsi.astype(complex), np.zeros((n, nc))], [np.zeros((nc, n)), np.eye(nc)]])
    sig = linalg.eigvals(K, W)
    sig = sig[np.isfinite(sig)]
    return float(np.max(sig.real))


def growth_rate_sugar(k, H, nu, A, kappa, vs, cbar_fn, gS=0.0, Ds=0.0, Sbar_fn=None, phi0=0.0, m=400):
    """Largest real part of sigma(k) with the sugar scalar (Sec. 3.2, the full x = (psi, omega,
    S, phi) problem with omega eliminated), in the lattice form of the model:
        F_y = -A c - gS S (1 - phi0 c)                     (A = g R, gS = g S*)
        sigma M psi = nu M^2 psi + i k [(A - gS phi0 Sbar) c + gS (1 - phi0 cbar) S]
        sigma c     = i k cbar' psi + (Vs D + kappa M) c
        sigma S     = i k Sbar' psi + Ds M S
    x = (psi, c, S); clamped psi, Neumann c and S, as in ``growth_rate``.  Vs is constant in
    the linearisation (the paper drops the -phi div(Vs e_z) term, Sec. 3.1)."""
    h = H / m
    y = np.linspace(0.0, H, m + 1)
    n = m - 1
    D2 = (np.diag(-2.0 * np.ones(n)) + np.diag(np.ones(n - 1), 1) + np.diag(np.ones(n - 1), -1)) / h**2
    D4 = (np.diag(6.0 * np.ones(n)) + np.diag(-4.0 * np.ones(n - 1), 1) + np.diag(-4.0 * np.ones(n - 1), -1)
          + np.diag(np.ones(n - 2), 2) + np.diag(np.ones(n - 2), -2))
    D4[0, 0] += 1.0
    D4[-1, -1] += 1.0
    D4 /= h**4
    I = np.eye(n)
    Mpsi = D2 - k**2 * I
    M2psi = D4 - 2.0 * k**2 * D2 + k**4 * I
    nc = m + 1
    Dc = np.zeros((nc, nc))
    D2c = np.zeros((nc, nc))
    for j in range(nc):
        jm, jp = j - 1, j + 1
        if jm < 0:
            jm = 1
        if jp > m:
            jp = m - 1
        if 0 < j < m:
            Dc[j, jp] += 0.5 / h
            Dc[j, jm] -= 0.5 / h
        D2c[j, jp] += 1.0 / h**2
        D2c[j, jm] += 1.0 / h**2
        D2c[j, j] -= 2.0 / h**2
    Mc = D2c - k**2 * np.eye(nc)
    cb = cbar_fn(y)
    Sb = Sbar_fn(y) if Sbar_fn is not None else np.zeros_like(y)
    dcb = np.gradient(cb, y)
    dSb = np.gradient(Sb, y)
    Aeff = A - gS * phi0 * Sb        # coefficient of c in -F_y
    Beff = gS * (1.0 - phi0 * cb)    # coefficient of S in -F_y
    Cpc = np.zeros((n, nc), dtype=complex)
    Cpc[:, 1:-1] = 1j * k * np.diag(Aeff[1:-1])
    CpS = np.zeros((n, nc), dtype=complex)
    CpS[:, 1:-1] = 1j * k * np.diag(Beff[1:-1])
    Ccp = np.zeros((nc, n), dtype=complex)
    Ccp[1:-1, :] = 1j * k * np.diag(dcb[1:-1])
    CSp = np.zeros((nc, n), dtype=complex)
    CSp[1:-1, :] = 1j * k * np.diag(dSb[1:-1])
    Z = np.zeros((nc, nc))
    K = np.block([[nu * M2psi.astype(complex), Cpc, CpS],
                  [Ccp, (vs * Dc + kappa * Mc).astype(complex), Z],
                  [CSp, Z, (Ds * Mc).astype(complex)]])
    W = np.block([[Mpsi.astype(complex), np.zeros((n, nc)), np.zeros((n, nc))],
                  [np.zeros((nc, n)), np.eye(nc), Z],
                  [np.zeros((nc, n)), Z, np.eye(nc)]])
    sig = linalg.eigvals(K, W)
    sig = sig[np.isfinite(sig)]
    return float(np.max(sig.real))


def front_height(c, level=0.5):
    """Front position per column (Sec. 4.1): lowest height where c reaches `level`,
    scanning up from the floor, linearly interpolated; node v sits at height v + 1/2.
    c is indexed [y][x]."""
    ny, nx = c.shape
    out = np.empty(nx)
    for x in range(nx):
        col = c[:, x]
        j = int(np.argmax(col >= level))
        if j == 0:
            out[x] = 0.5
        else:
            f = (level - col[j - 1]) / (col[j] - col[j - 1])
            out[x] = (j - 1) + f + 0.5
    return out
