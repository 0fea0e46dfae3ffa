"""Scattering states by mode matching: an independent route to the quantities
the oracle computes from Green functions.

Instead of inverting E - H - Sigma, the stationary Schrodinger equation
(E - H) psi = 0 is solved on the system with the wave function in every lead
written as incoming plus outgoing Bloch modes of the clean lead (the
Landauer-Buttiker scattering picture that Sec. 2.3's formula for T_kl
expresses through G).  The outgoing amplitudes give the scattering matrix;
|S|^2, the eigenvalues of t^dagger t, and the injected densities |psi|^2 / v
follow without any Green function.  Used only by tests, to pin the oracle.

Two geometries:

* slice systems with clean square leads of width M, hopping t (transverse
  modes phi_m(y) = sqrt(2/(M+1)) sin(m pi y/(M+1)), energies 2 t cos(m pi/(M+1)));
* site graphs with one-dimensional chain leads, lead p attached to one site.

For a lead mode with transverse energy e_m, the cell-to-cell factor lambda
solves lambda^2 - z lambda + 1 = 0, z = (E - e_m)/t.  The outgoing root is the
one that decays away from the system at E + i0 (retarded); the incoming one is
its inverse.  With c_m(j) = a lambda_in^j + b lambda_out^j on lead cell j = 1,
2, ..., the equation of lead cell 1 reduces to continuity with the system's
end cell: <phi_m | psi_end> = a + b.  A mode is open when |lambda| = 1; its
velocity is |t| |lambda - 1/lambda|.
"""
import numpy as np


def _mode_roots(E, e, t):
    """(lambda_out, lambda_in, open) of a lead mode with transverse energy e."""
    z = (E - e) / t
    r = np.roots([1.0, -(E + 1e-9j - e) / t, 1.0])
    ret = r[np.argmin(np.abs(r))]            # decays into the lead at E + i0
    r0 = np.roots([1.0, -complex(z), 1.0])
    lo = r0[np.argmin(np.abs(r0 - ret))]
    is_open = abs(z) < 2.0
    if is_open:
        lo = lo / abs(lo)
    return lo, 1.0 / lo, is_open


def square_lead_modes(M, t, E):
    y = np.arange(1, M + 1)
    m = np.arange(1, M + 1)
    phi = np.sqrt(2.0 / (M + 1)) * np.sin(np.outer(y, m) * np.pi / (M + 1))
    e = 2.0 * t * np.cos(m * np.pi / (M + 1))
    lo = np.empty(M, complex)
    li = np.empty(M, complex)
    op = np.zeros(M, bool)
    for k in range(M):
        lo[k], li[k], op[k] = _mode_roots(E, e[k], t)
    v = np.abs(t) * np.abs(lo - 1.0 / lo)
    return phi, lo, li, op, v


def slice_system_scattering(H0, V, eps, L, E, t):
    """Scattering solution of a slice system between two clean square leads
    of width M, hopping t (V = t I inside the system and to the leads).

    Returns dict with
      t, r : transmission / reflection amplitude matrices for injection from
             the left, flux-normalised, restricted to open modes (t[m, n]: out
             mode m on the right, in mode n on the left);
      T    : sum |t|^2;
      psiL : (n_open, L, M) left-injected scattering states (unit incoming
             amplitude) on the system, vL their velocities;
      psiR, vR : the same for injection from the right."""
    H0 = np.asarray(H0, complex)
    M = H0.shape[0]
    assert np.allclose(V, t * np.eye(M))
    phi, lo, li, op, v = square_lead_modes(M, t, E)
    N = M * L
    nu = N + 2 * M
    A = np.zeros((nu, nu), complex)
    # system rows: (E - H_n) psi_n - t psi_{n-1} - t psi_{n+1} = 0
    for n in range(L):
        blk = slice(n * M, (n + 1) * M)
        A[blk, blk] = E * np.eye(M) - H0 - (np.diag(eps[n]) if eps is not None else 0)
        if n > 0:
            A[blk, (n - 1) * M:n * M] = -t * np.eye(M)
        if n + 1 < L:
            A[blk, (n + 1) * M:(n + 2) * M] = -t * np.eye(M)
    # lead cell 1 enters slice 0 (left) and slice L-1 (right): -t phi (a li + b lo)
    bl, br = slice(N, N + M), slice(N + M, N + 2 * M)
    A[0:M, bl] = -t * phi * lo[None, :]
    A[N - M:N, br] += -t * phi * lo[None, :]
    # continuity rows: phi^T psi_end - b = a
    A[bl, 0:M] = phi.T
    A[bl, bl] = -np.eye(M)
    A[br, N - M:N] = phi.T
    A[br, br] = -np.eye(M)

    def solve(side, n):
        rhs = np.zeros(nu, complex)
        rows = slice(0, M) if side == 0 else slice(N - M, N)
        rhs[rows] += t * phi[:, n] * li[n]     # known incoming part, moved right
        rhs[(bl if side == 0 else br).start + n] = 1.0
        x = np.linalg.solve(A, rhs)
        return x[:N].reshape(L, M), x[bl], x[br]

    openm = np.flatnonzero(op)
    psiL, psiR = [], []
    tm = np.zeros((len(openm), len(openm)), complex)
    rm = np.zeros_like(tm)
    for c, n in enumerate(openm):
        psi, bL, bR = solve(0, n)
        psiL.append(psi)
        tm[:, c] = bR[openm] * np.sqrt(v[openm] / v[n])
        rm[:, c] = bL[openm] * np.sqrt(v[openm] / v[n])
        psi, _, _ = solve(1, n)
        psiR.append(psi)
    return dict(t=tm, r=rm, T=float(np.sum(np.abs(tm) ** 2)),
                psiL=np.array(psiL).reshape(len(openm), L, M), vL=v[openm],
                psiR=np.array(psiR).reshape(len(openm), L, M), vR=v[openm])


def graph_scattering(H, E, lead_site, t, want_states=False):
    """Scattering matrix S[k, l] (flux-normalised; all leads alike) of a site
    graph with one-dimensional chain leads of hopping t, lead p attached by
    hopping t to site lead_site[p].  Requires |E| < 2|t| (one open mode).
    With want_states also the scattering states psi[l] (unit incoming
    amplitude in lead l) on the graph's sites and the lead velocity."""
    H = np.asarray(H, complex)
    N = H.shape[0]
    P = len(lead_site)
    lo, li, op = _mode_roots(E, 0.0, t)
    assert op, "the chain leads must be open at E"
    A = np.zeros((N + P, N + P), complex)
    A[:N, :N] = E * np.eye(N) - H
    for p, s in enumerate(lead_site):
        A[s, N + p] += -t * lo
        A[N + p, s] = 1.0
        A[N + p, N + p] = -1.0
    S = np.zeros((P, P), complex)
    psi = np.zeros((P, N), complex)
    for l, s in enumerate(lead_site):
        rhs = np.zeros(N + P, complex)
        rhs[s] += t * li
        rhs[N + l] = 1.0
        x = np.linalg.solve(A, rhs)
        S[:, l] = x[N:]
        psi[l] = x[:N]
    if want_states:
        return S, psi, abs(t) * abs(lo - 1.0 / lo)
    return S


def lead_surface_g_from_modes(H0, V, z, side):
    """Retarded surface Green function of a general lead at complex energy
    z = E + i eta from its Bloch modes (no decimation).  Left lead (side 0):
    cell j + 1 lies outward of cell j with H_{j, j+1} = V, so a mode
    psi_j = u lambda^j solves (z - H0 - lambda V - V^dagger / lambda) u = 0;
    the m modes that decay outward at Im z > 0 (|lambda| < 1) give the Bloch
    matrix F = U Lambda U^{-1} with psi_{j+1} = F psi_j, and eliminating
    every outer cell leaves g = (z - H0 - V F)^{-1}.  Right lead (side 1):
    V and V^dagger exchange roles.  A singular V (a graphene ribbon's
    two-slice cell) is fine: its modes with lambda = 0 are among the m, as
    long as their U is invertible."""
    import scipy.linalg as sla
    H0 = np.asarray(H0, complex)
    V = np.asarray(V, complex)
    m = H0.shape[0]
    Vo, Vi = (V, V.conj().T) if side == 0 else (V.conj().T, V)
    I, Z = np.eye(m), np.zeros((m, m))
    # lambda [[I, 0], [0, Vo]] y = [[0, I], [-Vi, z - H0]] y, y = [u; lambda u]
    A = np.block([[Z, I], [-Vi, z * I - H0]])
    B = np.block([[I, Z], [Z, Vo]])
    lam, Y = sla.eig(A, B)
    out = np.flatnonzero(np.abs(lam) < 1.0)
    assert len(out) == m, "a retarded lead has as many outgoing modes as orbitals"
    U = Y[:m, out]
    F = U @ np.diag(lam[out]) @ np.linalg.inv(U)
    return np.linalg.inv(z * I - H0 - Vo @ F)


def lead_modes(H0, V, E, side, eta=1e-9):
    """Bloch modes of a general lead at real energy E, split into the m
    outgoing ones (decaying outward at E + i eta, or propagating outward) and
    the propagating incoming ones.  Cells j = 0, 1, ... run outward with
    H_{j, j+1} = Vo (V for the left lead, V^dagger for the right one); a mode
    is psi_j = u lambda^j with (E - H0 - lambda Vo - Vo^dagger / lambda) u = 0
    and |u| = 1, and carries the outward current -2 Im(lambda u^dagger Vo u)
    when |lambda| = 1.  Needs an invertible V and non-degenerate propagating
    modes.  Returns (lam_out, U_out, v_out, lam_in, U_in, v_in) with v the
    absolute currents (zero for evanescent outgoing modes)."""
    import scipy.linalg as sla
    H0 = np.asarray(H0, complex)
    V = np.asarray(V, complex)
    m = H0.shape[0]
    Vo, Vi = (V, V.conj().T) if side == 0 else (V.conj().T, V)
    I, Z = np.eye(m), np.zeros((m, m))

    def pencil(z):
        lam, Y = sla.eig(np.block([[Z, I], [-Vi, z * I - H0]]), np.block([[I, Z], [Z, Vo]]))
        U = Y[:m] / np.linalg.norm(Y[:m], axis=0)
        return lam, U

    lam_c, _ = pencil(E + 1j * eta)
    lam, U = pencil(E)
    # pair every real-E mode with its shifted copy
    used, out, inn = set(), [], []
    for k in range(2 * m):
        j = min((i for i in range(2 * m) if i not in used), key=lambda i: abs(lam_c[i] - lam[k]))
        used.add(j)
        (out if abs(lam_c[j]) < 1.0 else inn).append(k)
    assert len(out) == m
    cur = -2 * np.imag(lam * np.einsum("im,ij,jm->m", U.conj(), Vo, U))
    prop = np.abs(np.abs(lam) - 1.0) < 1e-7
    v_out = np.where(prop[out], np.abs(cur[out]), 0.0)
    inn = [k for k in inn if prop[k]]
    return lam[out], U[:, out], v_out, lam[inn], U[:, inn], np.abs(cur[inn])


def slice_system_scattering_general(H0, V, eps, L, E, leads):
    """T of a slice system (H_{n, n-1} = V, slices H0 + diag(eps_n)) between
    two general leads leads[p] = (H0_p, V_p) that continue it (left cells to
    the left with the same orientation, right cells to the right), by mode
    matching: the system's end slice equals the lead wave continued one cell
    inward.  Returns (T, R) summed over propagating modes, flux-normalised."""
    H0 = np.asarray(H0, complex)
    M = H0.shape[0]
    N = M * L
    modes = [lead_modes(*leads[p], E, p) for p in (0, 1)]
    nu = N + 2 * M
    A = np.zeros((nu, nu), complex)
    for n in range(L):
        b = slice(n * M, (n + 1) * M)
        A[b, b] = E * np.eye(M) - H0 - (np.diag(eps[n]) if eps is not None else 0)
        if n > 0:
            A[b, (n - 1) * M:n * M] = -V
        if n + 1 < L:
            A[b, (n + 1) * M:(n + 2) * M] = -V.conj().T
    rows = [slice(0, M), slice(N - M, N)]
    cols = [slice(N, N + M), slice(N + M, N + 2 * M)]
    Vo = [np.asarray(leads[0][1], complex), np.asarray(leads[1][1], complex).conj().T]
    for p in (0, 1):
        lo, Uo = modes[p][0], modes[p][1]
        # the end slice couples to lead cell 0 through Vo: -Vo psi_cell0
        A[rows[p], cols[p]] = -Vo[p] @ Uo
        # matching: psi_end - sum_m b_m u_m / lambda_m = (incoming part)
        A[cols[p], rows[p]] = np.eye(M)
        A[cols[p], cols[p]] = -Uo / lo[None, :]
    lo0, Uo0, vo0, li0, Ui0, vi0 = modes[0]
    T = R = 0.0
    for n in range(len(li0)):
        rhs = np.zeros(nu, complex)
        a = Ui0[:, n] / np.sqrt(vi0[n])
        rhs[rows[0]] = Vo[0] @ a
        rhs[cols[0]] = a / li0[n]
        x = np.linalg.solve(A, rhs)
        bL, bR = x[cols[0]], x[cols[1]]
        T += np.sum(np.abs(bR) ** 2 * modes[1][2])
        R += np.sum(np.abs(bL) ** 2 * vo0)
    return T, R, len(li0)
