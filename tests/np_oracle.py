"""A second, independently written restatement of the axisymmetric Shan-Chen step
(arXiv:1310.1871) in vectorised NumPy, used only to cross-check the C++ oracle
on tiny grids.  It is written from the paper's equations in array form (shifted
copies of ghost-padded fields) rather than site loops, so that a transcription
slip in either version shows up as a disagreement.

Fields are [Nr, Nz] (row = radial index, r_j = j + 1/2 + r_off; column = axial
index).
"""
import numpy as np

# D2Q9 velocities (c_z, c_r) and weights, App. A.
C = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)])
Wt = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
CS2 = 1.0 / 3.0


def _index_maps(Nr, Nz, g, zbc, rlo, wall):
    """Source row / column of every cell of a field padded by g, with the kind
    of ghost each row is: 'in' (real), 'half' (mirror about a mid-grid
    boundary: the axis or a wall) or 'node' (mirror about an inlet or outlet
    row)."""
    rows, kinds = [], []
    for jj in range(-g, Nr + g):
        if jj < 0:
            rows.append(-jj if rlo == 1 else -1 - jj)
            kinds.append('node' if rlo == 1 else 'half')
        elif jj >= Nr:
            rows.append(2 * (Nr - 1) - jj if wall == 2 else 2 * Nr - 1 - jj)
            kinds.append('node' if wall == 2 else 'half')
        else:
            rows.append(jj)
            kinds.append('in')
    ks = np.arange(-g, Nz + g)
    if zbc == 1:
        cols = np.where(ks < 0, -1 - ks, np.where(ks >= Nz, 2 * Nz - 1 - ks, ks))
        colsgn = np.where((ks < 0) | (ks >= Nz), -1.0, 1.0)
    else:
        cols = ks % Nz
        colsgn = np.ones(ks.size)
    return rows, kinds, cols, colsgn


def _pad(a, g, sgn_axis=1.0, sgn_wall=1.0, zbc=0, rlo=0, wall=0, velocity=False):
    """Ghost-pad a [Nr, Nz] field by g.  Columns: periodic, or mirrored about the
    z walls (a velocity changes sign there: no-slip).  Rows: mirrored with the
    given parity about the axis (bottom) and the outer wall (top); beyond an
    inlet or outlet row a scalar is mirrored about that row and a velocity
    continued linearly, 2 a(b) - a(b + m)."""
    Nr, Nz = a.shape
    rows, kinds, cols, colsgn = _index_maps(Nr, Nz, g, zbc, rlo, wall)
    ext = a[:, cols] * (colsgn if velocity else 1.0)  # real rows, padded columns
    out = np.empty((Nr + 2 * g, Nz + 2 * g))
    for t, jj in enumerate(range(-g, Nr + g)):
        if kinds[t] == 'in':
            out[t] = ext[jj]
        elif kinds[t] == 'half':
            out[t] = (sgn_axis if jj < 0 else sgn_wall) * ext[rows[t]]
        elif velocity:
            b = 0 if jj < 0 else Nr - 1
            out[t] = 2 * ext[b] - ext[rows[t]]
        else:
            out[t] = ext[rows[t]]
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


def _d1(p, g, Nr, Nz, comp):
    """1D 4th-order central difference along comp (0 = z, 1 = r), Sec. II.D."""
    dz, dr = (1, 0) if comp == 0 else (0, 1)
    return (8 * (_shift(p, g, dz, dr, Nr, Nz) - _shift(p, g, -dz, -dr, Nr, Nz))
            - (_shift(p, g, 2 * dz, 2 * dr, Nr, Nz) - _shift(p, g, -2 * dz, -2 * dr, Nr, Nz))) / 12.0


def step(f, tau, G, rho0=1.0, gz=0.0, wall=0, axisym=1, src_mode=0, zbc=0, rlo=0, r_off=0.0,
         rho_out=1.0, inlet=None, forcing=0):
    """One timestep.  wall: 0 free-slip, 1 no-slip, 2 outlet row; zbc: 0
    periodic, 1 no-slip z walls; rlo: 0 axis, 1 inlet row with velocity
    inlet = (u_z, u_r) per column; r_j = j + 1/2 + r_off; forcing: 0 the
    Shan-Chen velocity shift, 1 Guo, Zheng & Shi (2002)."""
    Q, Nr, Nz = f.shape
    r = (np.arange(Nr) + 0.5 + r_off)[:, None] * np.ones((1, Nz))
    rho = f.sum(0)
    jz = np.tensordot(C[:, 0].astype(float), f, 1)
    jr = np.tensordot(C[:, 1].astype(float), f, 1)
    psi = rho0 * (1 - np.exp(-rho / rho0))
    gp = 6
    bc = dict(zbc=zbc, rlo=rlo, wall=wall)
    P = _pad(psi, gp, **bc)
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
        UZ = _pad(uz, 2, 1.0, -1.0 if wall == 1 else 1.0, velocity=True, **bc)
        UR = _pad(ur, 2, -1.0, -1.0, velocity=True, **bc)
        druz = _d1(UZ, 2, Nr, Nz, 1)
        dzur = _d1(UR, 2, Nr, Nz, 0)
        drur = _d1(UR, 2, Nr, Nz, 1)
        mu = rho * CS2 * (tau - 0.5)
        S = -rho * ur / r
        Hz = (mu * (druz + dzur) - rho * ur * uz) / r
        Hr = (2 * mu * (drur - ur / r) - rho * ur * ur) / r
        for i in range(9):
            h[i] = Wt[i] * (S + (C[i, 0] * Hz + C[i, 1] * Hr) / CS2)
    if forcing == 1:
        # Guo: the equilibrium at u and the discrete force
        # (1 - 1/(2 tau)) W_i [(c_i - u)/c_s^2 + (c_i . u) c_i / c_s^4] . F
        ex, ey = C[:, 0, None, None].astype(float), C[:, 1, None, None].astype(float)
        force = Wt[:, None, None] * (((ex - uz) * Fz + (ey - ur) * Fr) / CS2
                                     + (ex * uz + ey * ur) * (ex * Fz + ey * Fr) / CS2 ** 2)
        post = f - (f - equilibrium(rho, uz, ur)) / tau + (1 - 1 / (2 * tau)) * force
    else:
        cu = C[:, 0, None, None] * vz + C[:, 1, None, None] * vr
        feq = Wt[:, None, None] * rho * (1 + 3 * cu + 4.5 * cu ** 2 - 1.5 * (vz ** 2 + vr ** 2))
        post = f - (f - feq) / tau
    # inlet / outlet rows: the equilibrium of the imposed density and velocity,
    # without source, is what leaves them and what they hold next
    bnd = np.zeros(Nr, dtype=bool)
    if rlo == 1:
        post[:, 0] = equilibrium(rho[1:2], np.asarray(inlet[0], float)[None],
                                 np.asarray(inlet[1], float)[None])[:, 0]
        h[:, 0] = 0.0
        bnd[0] = True
    if wall == 2:
        post[:, Nr - 1] = equilibrium(np.full((1, Nz), rho_out), uz[Nr - 2:Nr - 1],
                                      ur[Nr - 2:Nr - 1])[:, 0]
        h[:, Nr - 1] = 0.0
        bnd[Nr - 1] = True
    # streaming: push every population along its link, then patch the walls
    new = np.empty_like(f)
    rev = {0: 0, 1: 3, 2: 4, 3: 1, 4: 2, 5: 7, 6: 8, 7: 5, 8: 6}
    mir = {0: 0, 1: 1, 2: 4, 3: 3, 4: 2, 5: 8, 6: 7, 7: 6, 8: 5}
    for i in range(9):
        cz, cr = C[i]
        for j in range(Nr):
            for k in range(Nz):
                if bnd[j]:
                    new[i, j, k] = post[i, j, k]
                    continue
                sj, sk, si = j - cr, (k - cz) % Nz, i
                if zbc == 1 and not 0 <= k - cz < Nz:
                    sj, sk, si = j, k, rev[i]
                elif sj < 0:
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
