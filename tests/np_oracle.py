"""A second, independently written restatement of the axisymmetric Shan-Chen step
(arXiv:1310.1871) in vectorised NumPy, used only to cross-check the C++ oracle
on tiny grids.  It is written from the paper's equations in array form (shifted
copies of ghost-padded fields) rather than site loops, so that a transcription
slip in either version shows up as a disagreement.

Fields are [Nr, Nz] (row = radial index, r_j = j + 1/2; column = axial index).
"""
import numpy as np

# D2Q9 velocities (c_z, c_r) and weights, App. A.
C = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)])
Wt = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CS2 = 1.0 / 3.0


def _pad(a, g, sgn_axis=1.0, sgn_wall=1.0):
    """Ghost-pad a [Nr, Nz] field by g: periodic in z, mirrored in r with the
    given parity at the axis (bottom) and at the outer wall (top)."""
    Nr, Nz = a.shape
    out = np.empty((Nr + 2 * g, Nz + 2 * g))
    cols = np.arange(-g, Nz + g) % Nz
    for jj in range(-g, Nr + g):
        if jj < 0:
            row, s = -1 - jj, sgn_axis
        elif jj >= Nr:
            row, s = 2 * Nr - 1 - jj, sgn_wall
        else:
            row, s = jj, 1.0
        out[jj + g] = s * a[row, cols]
    return out


def _shift(p, g, dz, dr, Nr, Nz):
    """View of padded field p at offset (dz, dr) over the [Nr, Nz] interior."""
    return p[g + dr: g + dr + Nr, g + dz: g + dz + Nz]


def _iso(p, g, Nr, Nz, comp):
    """Isotropic 4th-order derivative along comp (0 = z, 1 = r), Sec. II.D."""
    acc = np.zeros((Nr, Nz))
    for (cz, cr) in C[1:]:
        c = (cz, cr)[comp]
        if c == 0:
            continue
        acc += c * (8 * _shift(p, g, cz, cr, Nr, Nz) - _shift(p, g, 2 * cz, 2 * cr, Nr, Nz))
    return acc / 36.0


def step(f, tau, G, rho0=1.0, gz=0.0, wall=0, axisym=1, src_mode=0):
    Q, Nr, Nz = f.shape
    r = (np.arange(Nr) + 0.5)[:, None] * np.ones((1, Nz))
    rho = f.sum(0)
    jz = np.tensordot(C[:, 0].astype(float), f, 1)
    jr = np.tensordot(C[:, 1].astype(float), f, 1)
    psi = rho0 * (1 - np.exp(-rho / rho0))
    gp = 6
    P = _pad(psi, gp)
    # Shan-Chen force (radius-1, weighted).
    sz = sum(Wt[i] * C[i, 0] * _shift(P, gp, *C[i], Nr, Nz) for i in range(1, 9))
    sr = sum(Wt[i] * C[i, 1] * _shift(P, gp, *C[i], Nr, Nz) for i in range(1, 9))
    Fz = -G * psi * sz
    Fr = -G * psi * sr
    if axisym:
        # d_r psi on an extended window (real rows plus 2 ghost rows each side),
        # evaluated straight from the mirror-padded psi.
        Dr_ext = np.zeros((Nr + 4, Nz + 4))
        D1_ext = np.zeros((Nr + 4, Nz + 4))
        for a in range(Nr + 4):
            for b in range(Nz + 4):
                jj, kk = a - 2 + gp, b - 2 + gp
                s = 0.0
                for (cz, cr) in C[1:]:
                    if cr:
                        s += cr * (8 * P[jj + cr, kk + cz] - P[jj + 2 * cr, kk + 2 * cz])
                Dr_ext[a, b] = s / 36.0
                D1_ext[a, b] = (-P[jj + 2, kk] + 8 * P[jj + 1, kk] - 8 * P[jj - 1, kk] + P[jj - 2, kk]) / 12.0
        Dr = Dr_ext[2:-2, 2:-2]
        Drr = _iso(Dr_ext, 2, Nr, Nz, 1)
        Dzr = (-D1_ext[2:-2, 4:] + 8 * D1_ext[2:-2, 3:-1] - 8 * D1_ext[2:-2, 1:-3] + D1_ext[2:-2, :-4]) / 12.0
        Fz = Fz - (G / 2) * CS2 * CS2 * psi * Dzr / r
        Fr = Fr - (G / 2) * CS2 * CS2 * psi * (Drr / r - Dr / r ** 2)
    Fz = Fz + rho * gz
    uz, ur = (jz + Fz / 2) / rho, (jr + Fr / 2) / rho
    vz, vr = (jz + tau * Fz) / rho, (jr + tau * Fr) / rho
    h = np.zeros_like(f)
    if axisym:
        UZ = _pad(uz, 2, 1.0, -1.0 if wall == 1 else 1.0)
        UR = _pad(ur, 2, -1.0, -1.0)
        druz = _iso(UZ, 2, Nr, Nz, 1)
        dzur = _iso(UR, 2, Nr, Nz, 0)
        drur = _iso(UR, 2, Nr, Nz, 1)
        mu = rho * CS2 * (tau - 0.5)
        S = -rho * ur / r
        Hz = (mu * (druz + dzur) - rho * ur * uz) / r
        Hr = (2 * mu * (drur - ur / r) - rho * ur * ur) / r
        for i in range(9):
            h[i] = Wt[i] * (S + (C[i, 0] * Hz + C[i, 1] * Hr) / CS2)
    cu = C[:, 0, None, None] * vz + C[:, 1, None, None] * vr
    feq = Wt[:, None, None] * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (vz ** 2 + vr ** 2))
    post = f - (f - feq) / tau
    # streaming: push every population along its link, then patch the walls
    new = np.empty_like(f)
    rev = {0: 0, 1: 3, 2: 4, 3: 1, 4: 2, 5: 7, 6: 8, 7: 5, 8: 6}
    mir = {0: 0, 1: 1, 2: 4, 3: 3, 4: 2, 5: 8, 6: 7, 7: 6, 8: 5}
    for i in range(9):
        cz, cr = C[i]
        for j in range(Nr):
            for k in range(Nz):
                sj, sk, si = j - cr, (k - cz) % Nz, i
                if sj < 0:
                    sj, si = 0, mir[i]
                elif sj >= Nr:
                    if wall == 1:
                        sj, sk, si = Nr - 1, k, rev[i]
                    else:
                        sj, si = Nr - 1, mir[i]
                if src_mode == 1:  # link average
                    new[i, j, k] = post[si, sj, sk] + 0.5 * (h[si, sj, sk] + h[i, j, k])
                else:  # departure-site value
                    new[i, j, k] = post[si, sj, sk] + h[si, sj, sk]
    return new


def equilibrium(rho, uz, ur):
    cu = C[:, 0, None, None] * uz + C[:, 1, None, None] * ur
    return Wt[:, None, None] * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (uz ** 2 + ur ** 2))
