"""Plain, slow, FP64 CPU oracle of the OkMC-with-exact-elasticity hot path.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use this module.
It shares no code with the CUDA path and imports nothing from it.

What it computes, in the paper's order (Santos-Gueemes, Ortiz, Segurado,
"An FFT based approach to account for elastic interactions in OkMC"):

1. Defect eigenstrains (Sec. 3.1, Eq. eig_shearloop for prismatic loops; the
   point-defect eigenstrain from the relaxation volume, Sec. 3.1) rasterised on
   the voxel grid of Sec. 3.4 (voxel centres x_k = (L/N)(1/2 + n_k)).
2. The periodic elastic problem with eigenstrain (Sec. 3.2, Eqs.
   EIG_elastic_real / EIG_elastic_fourier / basicgammacomplete / summaryEL),
   solved by direct substitution in Fourier space on the discrete frequencies
   of Sec. 3.4 (Eq. frequencies).  The FFT is numpy's (a library primitive).
3. Interaction energies (Sec. 2, Eq. interaction_energy3), written as
   E_i(Y) = -int eps*_i(Y) : sigma^(-i) dV, with sigma^(-i) the stress of all
   defects except i.
4. The paper's translation of a defect's field by the shift theorem (Sec. 3.3, Eq.
   shift), the dipole approximation of the same energies (Sec. 2.1, Eq. interaction_energy4)
   (also for a point defect whose dipole tensor is given, Table 1)
   and dislocation lines by field dislocation mechanics (Sec. 3.2, Eqs. Nye2,
   eq_EIG_fourier, plastic_0): the Nye tensor of a line, the incompatible plastic
   distortion in Fourier space and its symmetric part as eigenstrain.
5. Rates (Sec. 5, Eqs. unbiased_boltzmann, biased_forward/backward_boltzmann),
   the frequency line and jump selection (Eqs. frequency_line, selection_jump),
   the fixed time step and Poisson event counts (Eqs. time_step, poisson;
   Appendix A, Algorithm 1), and a residence-time (one event per step) variant.

Readings where the paper is silent or ambiguous (each is repeated in the
repository's design notes):

* Green operator indices (Eq. basicgammacomplete is garbled): the standard
  form eps_hat = sym(m (x) K(m)^-1 (tau_hat . m)), K_ik = C_ijkl m_j m_l,
  tau_hat = C : eps*_hat, m = xi/|xi|; sigma_hat = C : (eps_hat - eps*_hat).
* Zero frequency: MEAN_STRESS_ZERO (sigma_hat(0) = 0) or MEAN_STRAIN_ZERO
  (eps_hat(0) = 0, hence sigma_hat(0) = -C : eps*_hat(0); Appendix B).
* Even grid edges: the Nyquist index uses n = -N/2 (Eq. frequencies) and the
  stress is the real part of the inverse transform (the field is real).
* Loop eigenstrain: slab |(x-X).n| <= h/2, in-plane radius <= R, 4x4x4
  subsamples per voxel, weights renormalised so that sum(w) V_vox equals the
  exact shape volume pi R^2 h; pure prismatic interstitial loop, n = b/|b|,
  eps* = sym(b (x) n)/h (Eq. eig_shearloop with e = h).
* SIA cluster of s atoms: sphere of radius r = max(h, (3 s Omega / 4 pi)^(1/3)),
  Omega = a0^3/2, dilatational eigenstrain with trace integral 1.5 s Omega.
* Lattice parameter a0 equals the voxel edge h; positions are integers in
  units of a0/2 on the bcc lattice (all even or all odd); the parity is the
  rasterisation class.
* Dislocation lines: the Burgers vector density of each sub-segment (at most h/4 long)
  is spread to the 8 surrounding voxel centres with trilinear weights; a loop's line
  runs clockwise seen from the tip of its oriented area A (so that curl U^p = -alpha,
  Eq. curlUe, holds with U^p = b (x) n on the loop's surface); a straight line is one
  period of a periodic line, whose net Burgers vector drops out with the xi = 0 term
  (a uniform compensating density); the compatible part of Eq. plastic_0 is a uniform
  distortion.
* Rates: nu_ij = (1/z_i) nu0 exp(-(E_m,i + (E_i(X+lambda_j) - E_i(X))/2)/k_B T)
  over the z_i allowed jumps (Eq. biased_forward_boltzmann generalised from
  z = 2 to z jumps).

Units: length nm, stress GPa, energy eV.
"""
from __future__ import annotations

import math

import numpy as np

PI = 3.141592653589793
KAPPA = 6.241509074            # eV per (GPa nm^3)
KB = 8.617333262e-5            # Boltzmann constant, eV/K
NU0_DEFAULT = 1.0e13           # attempt frequency, 1/s

LOOP_111, LOOP_100, SIA_CLUSTER = 0, 1, 2
IMMOBILE, ONE_D, THREE_D = 0, 1, 2
MEAN_STRESS_ZERO, MEAN_STRAIN_ZERO = 0, 1

AXES_111 = np.array([[1, 1, 1], [-1, 1, 1], [1, -1, 1], [1, 1, -1]], dtype=np.int64)
AXES_100 = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.int64)
# six independent components of a symmetric tensor, in this order
VOIGT = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
# jump j <-> lambda_j = (a0/2)(sx, sy, sz), j = 4 (sx>0) + 2 (sy>0) + (sz>0)
JUMPS = np.array([[1 if (j >> 2) & 1 else -1, 1 if (j >> 1) & 1 else -1, 1 if j & 1 else -1]
                  for j in range(8)], dtype=np.int64)


# --------------------------------------------------------------------------
# material (Table 1 and the isotropic reduction of Sec. 4)
# --------------------------------------------------------------------------
def stiffness_cubic(C11, C12, C44):
    """Full C_ijkl of a cubic crystal whose cube axes are the grid axes (Table 1)."""
    C = np.zeros((3, 3, 3, 3))
    for i in range(3):
        for j in range(3):
            for k in range(3):
                for l in range(3):
                    v = 0.0
                    if i == j and k == l:
                        v += C12
                    if i == k and j == l:
                        v += C44
                    if i == l and j == k:
                        v += C44
                    if i == j == k == l:
                        v += C11 - C12 - 2.0 * C44
                    C[i, j, k, l] = v
    return C


def isotropic_cubic_constants(mu, nu):
    """(C11, C12, C44) of an isotropic solid with shear modulus mu, Poisson ratio nu."""
    lam = 2.0 * mu * nu / (1.0 - 2.0 * nu)
    return lam + 2.0 * mu, lam, mu


def zener_isotropic_moduli(C11, C12):
    """Young's modulus and Poisson ratio of the Sec. 4 isotropic reduction
    (C11, C12 kept, C44 := (C11 - C12)/2)."""
    nu = C12 / (C11 + C12)
    E = (C11 - C12) * (C11 + 2.0 * C12) / (C11 + C12)
    return E, nu


def to_tensor(v6):
    """(6, ...) symmetric components -> (3, 3, ...) tensor."""
    v6 = np.asarray(v6)
    t = np.zeros((3, 3) + v6.shape[1:], dtype=v6.dtype)
    for a, (i, j) in enumerate(VOIGT):
        t[i, j] = v6[a]
        t[j, i] = v6[a]
    return t


def to_voigt6(t):
    """(3, 3, ...) symmetric tensor -> (6, ...) components."""
    return np.stack([t[i, j] for (i, j) in VOIGT])


def ddot6(a6, b6):
    """a : b for symmetric tensors held as 6 components (off-diagonals count twice)."""
    return (a6[0] * b6[0] + a6[1] * b6[1] + a6[2] * b6[2]
            + 2.0 * (a6[3] * b6[3] + a6[4] * b6[4] + a6[5] * b6[5]))


# --------------------------------------------------------------------------
# defects -> eigenstrain stencils (Sec. 3.1, Eq. eig_shearloop; Sec. 3.4 grid)
# --------------------------------------------------------------------------
def defect_geometry(d, h):
    """Shape, eigenstrain tensor e (3x3) and shape volume of one defect record."""
    t = int(d['type'])
    if t in (LOOP_111, LOOP_100):
        a = (AXES_111 if t == LOOP_111 else AXES_100)[int(d['axis'])]
        a2 = int(a @ a)
        n = a / math.sqrt(a2)
        blen = (math.sqrt(3.0) / 2.0) * h if t == LOOP_111 else h      # |b|, a0 = h
        R = float(d['radius_nm'])
        # eps* = sym(b (x) n)/e with b = |b| n and slab thickness e = h
        e = (blen / h) * np.outer(n, n)
        t_ = 8.0 * R / h
        return dict(kind='disk', a=a, a2=a2, n=n, b=blen * n, R=R,
                    Rq=float(a2) * (t_ * t_),
                    v_over_h3=PI * (R / h) ** 2,
                    extent=int(math.ceil(R / h)) + 2, e=e)
    if t == SIA_CLUSTER:
        s = int(d['size'])
        # sphere radius rho = r/h = max(1, (3 s Omega/(4 pi))^(1/3)) with Omega = h^3/2;
        # the inside test |x|^2 <= rho^2 is done on cubes: |x|^6 <= rho^6 (integers in h/8)
        q = 3.0 * s / (8.0 * PI)                          # rho^3 when rho > 1
        rho3 = q if q > 1.0 else 1.0
        T6 = 262144.0 * (rho3 * rho3)                      # (8 rho)^6
        v = (4.0 * PI / 3.0) * rho3                        # V_shape / h^3
        # trace of the integrated eigenstrain = relaxation volume 1.5 s Omega
        e = np.eye(3) * (1.5 * s * 0.5) / (3.0 * v)
        return dict(kind='sphere', s=s, T6=T6, v_over_h3=v,
                    extent=int(math.ceil(rho3 ** (1.0 / 3.0))) + 2, e=e)
    raise ValueError('unknown defect type %d' % t)


def stencil(d, cls, h):
    """Coverage stencil of defect d for rasterisation class cls (0 or 1).

    Returns (offsets (k, 3) int [dx, dy, dz] relative to the base voxel
    floor(pos/2), counts (k,) int in 1..64, alpha) with voxel weight
    w = count * alpha and sum(w) h^3 = shape volume.  Entries are sorted by
    (dz, dy, dx).  Subsample coordinates relative to the defect centre are
    integers in units of h/8: s = 8 v + 2 i + 1 - 4 cls, i = 0..3.
    """
    g = defect_geometry(d, h)
    E = g['extent']
    r = np.arange(-E, E + 1, dtype=np.int64)
    s1 = 8 * r[:, None] + 2 * np.arange(4, dtype=np.int64)[None, :] + 1 - 4 * cls   # (nv, 4)
    sx = s1[:, :, None, None, None, None]
    sy = s1[None, None, :, :, None, None]
    sz = s1[None, None, None, None, :, :]
    ss = sx * sx + sy * sy + sz * sz
    if g['kind'] == 'disk':
        a = g['a']
        sa = a[0] * sx + a[1] * sy + a[2] * sz
        inside = (sa * sa <= 16 * g['a2']) & ((g['a2'] * ss - sa * sa).astype(np.float64) <= g['Rq'])
    else:
        inside = (ss * ss * ss).astype(np.float64) <= g['T6']
    counts = inside.sum(axis=(1, 3, 5))            # [x, y, z]
    cz = np.transpose(counts, (2, 1, 0))            # [z, y, x]
    iz, iy, ix = np.nonzero(cz)
    offs = np.stack([r[ix], r[iy], r[iz]], axis=1)
    cnt = cz[iz, iy, ix].astype(np.int64)
    if np.any(np.abs(offs) == E):
        raise AssertionError('stencil reached its scan box edge')
    alpha = g['v_over_h3'] / float(cnt.sum())
    return offs, cnt, alpha


def base_voxel(pos):
    """Voxel that holds a defect at half-lattice position pos (floor(pos/2))."""
    return np.floor_divide(np.asarray(pos, dtype=np.int64), 2)


def pos_class(pos):
    p = np.asarray(pos, dtype=np.int64)
    c = int(p[0] & 1)
    if not np.all((p & 1) == c):
        raise ValueError('position %s is not a bcc site' % (p,))
    return c


def eigenstrain_field(defects, n, h, only=None, exclude=None, positions=None):
    """Sum of the voxelised eigenstrains, (6, nx, ny, nz) FP64 (Sec. 3.1, 3.4)."""
    n = tuple(int(v) for v in n)
    eps = np.zeros((6,) + n)
    flat = eps.reshape(6, -1)
    for i, d in enumerate(defects):
        if only is not None and i not in only:
            continue
        if exclude is not None and i in exclude:
            continue
        pos = np.asarray(d['pos'] if positions is None else positions[i], dtype=np.int64)
        c = pos_class(pos)
        offs, cnt, alpha = stencil(d, c, h)
        e6 = to_voigt6(defect_geometry(d, h)['e'])
        v = np.mod(base_voxel(pos)[None, :] + offs, np.array(n)[None, :])
        lin = np.ravel_multi_index((v[:, 0], v[:, 1], v[:, 2]), n)
        w = cnt * alpha
        for a in range(6):
            np.add.at(flat[a], lin, w * e6[a])
    return eps


# --------------------------------------------------------------------------
# periodic elastic solve (Sec. 3.2 and 3.4)
# --------------------------------------------------------------------------
def frequencies(N, L):
    """xi = 2 pi n / L with n from Eq. frequencies, in numpy's FFT index order."""
    return 2.0 * PI * (np.fft.fftfreq(N) * N) / L


def green_sigma_hat(C, xi, eps_hat_t, k0_mode, zero_mask):
    """sigma_hat = C:(Gamma_hat:(C:eps*_hat) - eps*_hat) at the given frequencies.

    xi: (..., 3) real; eps_hat_t: (3, 3, ...) complex; Eq. EIG_elastic_fourier,
    Eq. basicgammacomplete (standard index reading) and Eq. summaryEL.
    """
    tau = np.einsum('ijkl,kl...->ij...', C, eps_hat_t)
    nrm = np.sqrt(np.sum(xi * xi, axis=-1))
    safe = np.where(zero_mask, 1.0, nrm)
    m = xi / safe[..., None]
    K = np.einsum('ijkl,...j,...l->...ik', C, m, m)
    K = np.where(zero_mask[..., None, None], np.eye(3), K)
    v = np.einsum('ij...,...j->...i', tau, m)
    w = np.linalg.solve(K, v[..., None])[..., 0]                   # (..., 3)
    eps_c = 0.5 * (np.einsum('...i,...j->ij...', m, w) + np.einsum('...j,...i->ij...', m, w))
    sig = np.einsum('ijkl,kl...->ij...', C, eps_c) - tau
    if np.any(zero_mask):
        if k0_mode == MEAN_STRESS_ZERO:
            sig[:, :, zero_mask] = 0.0
        elif k0_mode == MEAN_STRAIN_ZERO:
            sig[:, :, zero_mask] = -tau[:, :, zero_mask]
        else:
            raise ValueError('k0_mode')
    return sig


def solve_stress(eps6, C, h, k0_mode=MEAN_STRESS_ZERO, dft=None):
    """Stress (6, nx, ny, nz) of the periodic eigenstrain field eps6 (same shape).

    Forward transform of eps*, the Green operator on every discrete frequency,
    inverse transform, real part.  ``dft`` may replace numpy's FFT by another
    transform pair (forward, inverse) acting on the last three axes.
    """
    fwd, inv = dft if dft is not None else (
        lambda a: np.fft.fftn(a, axes=(-3, -2, -1)),
        lambda a: np.fft.ifftn(a, axes=(-3, -2, -1)))
    n = eps6.shape[1:]
    L = [n[a] * h for a in range(3)]
    xs = [frequencies(n[a], L[a]) for a in range(3)]
    eh6 = fwd(eps6.astype(np.complex128))
    sh6 = np.empty_like(eh6)
    for ix in range(n[0]):                      # one x-slab at a time keeps memory small
        XI = np.stack(np.meshgrid(np.full(1, xs[0][ix]), xs[1], xs[2], indexing='ij'), axis=-1)[0]
        zero = np.all(XI == 0.0, axis=-1)
        sig = green_sigma_hat(C, XI, to_tensor(eh6[:, ix]), k0_mode, zero)
        sh6[:, ix] = to_voigt6(sig)
    return inv(sh6).real


def naive_dft_pair(n):
    """O(N^2) DFT along each of the last three axes, written out from the definition."""
    mats = []
    for N in n:
        j = np.arange(N)
        mats.append(np.exp(-2j * PI * np.outer(j, j) / N))

    def fwd(a):
        a = np.einsum('...xyz,ux->...uyz', a, mats[0])
        a = np.einsum('...xyz,vy->...xvz', a, mats[1])
        return np.einsum('...xyz,wz->...xyw', a, mats[2])

    def inv(a):
        a = np.einsum('...xyz,ux->...uyz', a, mats[0].conj()) / n[0]
        a = np.einsum('...xyz,vy->...xvz', a, mats[1].conj()) / n[1]
        return np.einsum('...xyz,wz->...xyw', a, mats[2].conj()) / n[2]
    return fwd, inv


# --------------------------------------------------------------------------
# interaction energies (Sec. 2, Eq. interaction_energy3; Sec. 3.3)
# --------------------------------------------------------------------------
def energy_of_stencil(d, pos_Y, sigma6, h):
    """-kappa V_vox sum_v eps*_d(Y)(v) : sigma(v) for defect d placed at pos_Y."""
    n = np.array(sigma6.shape[1:])
    c = pos_class(pos_Y)
    offs, cnt, alpha = stencil(d, c, h)
    e6 = to_voigt6(defect_geometry(d, h)['e'])
    v = np.mod(base_voxel(pos_Y)[None, :] + offs, n[None, :])
    sig = sigma6[:, v[:, 0], v[:, 1], v[:, 2]]          # (6, k)
    s = np.sum(cnt * alpha * ddot6(e6, sig))
    return -KAPPA * h ** 3 * s


def as_record(d):
    """Plain dict copy of a defect record (dict or numpy structured row)."""
    if isinstance(d, dict):
        return dict(d)
    return {k: (np.array(d[k]) if np.ndim(d[k]) else d[k].item()) for k in d.dtype.names}


def candidate_positions(pos):
    pos = np.asarray(pos, dtype=np.int64)
    return [pos + JUMPS[j] for j in range(8)]


def allowed_jumps(d):
    """Boolean mask over the 8 jumps for the defect's mobility (Sec. 5)."""
    mob = int(d['mobility'])
    if mob == IMMOBILE:
        return np.zeros(8, bool)
    if mob == THREE_D:
        return np.ones(8, bool)
    ax = AXES_111[int(d['axis'])]
    return np.array([np.array_equal(JUMPS[j], ax) or np.array_equal(JUMPS[j], -ax)
                     for j in range(8)])


def energies_bruteforce(defects, n, h, C, k0_mode=MEAN_STRESS_ZERO, dft=None):
    """E_i(X_i) and E_i(X_i + lambda_j) from the plain definition: one solve of all
    defects except i per defect (N_d + 1 solves in total counting the base field).
    Returns (E (n_d,), Ec (n_d, 8))."""
    nd = len(defects)
    E = np.zeros(nd)
    Ec = np.zeros((nd, 8))
    for i in range(nd):
        sig = solve_stress(eigenstrain_field(defects, n, h, exclude={i}), C, h, k0_mode, dft)
        E[i] = energy_of_stencil(defects[i], defects[i]['pos'], sig, h)
        for j, Y in enumerate(candidate_positions(defects[i]['pos'])):
            Ec[i, j] = energy_of_stencil(defects[i], Y, sig, h)
    return E, Ec


def energies_self_field(defects, n, h, C, k0_mode=MEAN_STRESS_ZERO, sample=None,
                        sigma_total=None):
    """Same quantities through sigma^(-i) = sigma - sigma_i (linearity); sigma_i is the
    solve of defect i alone.  ``sample`` limits the defects evaluated."""
    if sigma_total is None:
        sigma_total = solve_stress(eigenstrain_field(defects, n, h), C, h, k0_mode)
    idx = range(len(defects)) if sample is None else sample
    out = {}
    for i in idx:
        sig_i = solve_stress(eigenstrain_field(defects, n, h, only={i}), C, h, k0_mode)
        sig = sigma_total - sig_i
        e0 = energy_of_stencil(defects[i], defects[i]['pos'], sig, h)
        ec = np.array([energy_of_stencil(defects[i], Y, sig, h)
                       for Y in candidate_positions(defects[i]['pos'])])
        out[int(i)] = (e0, ec)
    return out, sigma_total


def self_term_table(d, n, h, C, k0_mode=MEAN_STRESS_ZERO):
    """W(c, k): energy of defect d's own stencil placed at the current position (k = 0)
    or at jump k-1 against the field of d alone at a reference site of class c.
    Translation invariance under whole-voxel shifts makes it position independent."""
    W = np.zeros((2, 9))
    for c in (0, 1):
        ref = np.array([c, c, c], dtype=np.int64)
        dd = as_record(d)
        dd['pos'] = ref
        sig = solve_stress(eigenstrain_field([dd], n, h), C, h, k0_mode)
        W[c, 0] = energy_of_stencil(d, ref, sig, h)
        for j, Y in enumerate(candidate_positions(ref)):
            W[c, 1 + j] = energy_of_stencil(d, Y, sig, h)
    return W


def green_operator_matrix(C, xi):
    """Gamma_hat(xi) as a map on symmetric tensors (3,3,3,3), extracted from the solve of
    Eq. EIG_elastic_fourier: for a polarisation tau, eps_hat = C^-1:sigma_hat + eps*_hat
    with eps*_hat = C^-1:tau."""
    C66 = stiffness_matrix(C)
    S66 = np.linalg.inv(C66)
    G = np.zeros((3, 3, 3, 3))
    for a, (k, l) in enumerate(VOIGT):
        tau6 = np.zeros(6)
        tau6[a] = 1.0
        tau = to_tensor(tau6)
        if k != l:
            tau = tau * 0.5            # unit symmetric tensor with tau_kl = tau_lk = 1/2
        epsstar = strain_from_engineering(S66 @ stress_vec(tau))
        sig = green_sigma_hat(C, np.asarray(xi, float)[None, :], epsstar[:, :, None].astype(complex),
                              MEAN_STRESS_ZERO, np.zeros(1, bool))[:, :, 0].real
        eps = strain_from_engineering(S66 @ stress_vec(sig)) + epsstar
        G[:, :, k, l] = eps
        G[:, :, l, k] = eps
    return G


# 6x6 helpers used only to invert C: stresses as plain VOIGT vectors, strains with
# engineering shears
def stress_vec(t):
    return np.array([t[0, 0], t[1, 1], t[2, 2], t[1, 2], t[0, 2], t[0, 1]])


def strain_from_engineering(v):
    return np.array([[v[0], v[5] / 2, v[4] / 2], [v[5] / 2, v[1], v[3] / 2], [v[4] / 2, v[3] / 2, v[2]]])


def stiffness_matrix(C):
    """6x6 stiffness acting on engineering strains, giving stresses in VOIGT order."""
    M = np.zeros((6, 6))
    for a, (i, j) in enumerate(VOIGT):
        for b, (k, l) in enumerate(VOIGT):
            M[a, b] = C[i, j, k, l]
    return M


def self_term_table_fourier(d, n, h, C, k0_mode=MEAN_STRESS_ZERO):
    """The table of ``self_term_table`` by Parseval: with w_c the count field of the
    class-c stencil placed at the origin, q(xi) = e : sigma_hat[e](xi) (the stress
    spectrum of a unit-amplitude eigenstrain e),
      W(c, 0)     = -kappa h^3 a_c^2 / N  sum_xi q |w_c|^2
      W(c, 1 + j) = -kappa h^3 a_c a_c' / N  Re sum_xi q conj(w_c') exp(+i xi.d_cj) w_c
    where c' = 1 - c and d_cj is the whole-voxel shift between the two stencils."""
    n = tuple(int(v) for v in n)
    N = n[0] * n[1] * n[2]
    e = defect_geometry(d, h)['e']
    e6 = to_voigt6(e)
    what, alpha = [], []
    for c in (0, 1):
        offs, cnt, a = stencil(d, c, h)
        f = np.zeros(n)
        v = np.mod(offs, np.array(n)[None, :])
        np.add.at(f, (v[:, 0], v[:, 1], v[:, 2]), cnt.astype(float))
        what.append(np.fft.fftn(f))
        alpha.append(a)
    xs = [frequencies(n[a], n[a] * h) for a in range(3)]
    fr = [np.fft.fftfreq(n[a]) * n[a] for a in range(3)]
    q = np.empty(n)
    for ix in range(n[0]):
        XI = np.stack(np.meshgrid(np.full(1, xs[0][ix]), xs[1], xs[2], indexing='ij'), axis=-1)[0]
        zero = np.all(XI == 0.0, axis=-1)
        eh = np.broadcast_to(e[:, :, None, None], (3, 3) + XI.shape[:2]).astype(complex)
        sig = green_sigma_hat(C, XI, eh, k0_mode, zero)
        q[ix] = ddot6(e6[:, None, None], to_voigt6(sig).real)
    W = np.zeros((2, 9))
    pref = -KAPPA * h ** 3 / N
    for c in (0, 1):
        cp = 1 - c
        W[c, 0] = pref * alpha[c] ** 2 * np.sum(q * np.abs(what[c]) ** 2)
        ref = np.array([c, c, c], dtype=np.int64)
        for j in range(8):
            dvec = base_voxel(ref + JUMPS[j]) - base_voxel(ref)
            ph = 2.0 * PI * (fr[0][:, None, None] * dvec[0] / n[0] + fr[1][None, :, None] * dvec[1] / n[1]
                             + fr[2][None, None, :] * dvec[2] / n[2])
            W[c, 1 + j] = pref * alpha[c] * alpha[cp] * np.sum(
                q * (np.conj(what[cp]) * np.exp(1j * ph) * what[c])).real
    return W


def unit_tensor(d, h):
    """(E, s) with the defect's eigenstrain e = s E and s its largest |component|:
    defects of one type and axis share E (the 1/2<111> and <100> loops per axis, the
    dilatational clusters), so a per-E kernel serves all of them."""
    e = defect_geometry(d, h)['e']
    s = float(np.abs(e).max())
    return e / s, s


def unit_kernel(E, n, h, C, k0_mode=MEAN_STRESS_ZERO):
    """Real-space kernel of a unit eigenstrain tensor E on the periodic grid,
    K(r) = (1/N) sum_xi Q(xi) exp(+i xi.r) with Q(xi) = E : sigma_hat[E](xi), the q of
    self_term_table_fourier for e = E (Eqs. EIG_elastic_fourier, basicgammacomplete,
    summaryEL on every discrete frequency).  Q is real and even, so only the real part
    of K enters the (symmetric, real) sums below: it is the real part of the inverse
    transform, the even-edge reading of the solve.  (nx, ny, nz) FP64."""
    n = tuple(int(v) for v in n)
    xs = [frequencies(n[a], n[a] * h) for a in range(3)]
    E6 = to_voigt6(E)
    Q = np.empty(n)
    for ix in range(n[0]):
        XI = np.stack(np.meshgrid(np.full(1, xs[0][ix]), xs[1], xs[2], indexing='ij'), axis=-1)[0]
        zero = np.all(XI == 0.0, axis=-1)
        eh = np.broadcast_to(E[:, :, None, None], (3, 3) + XI.shape[:2]).astype(complex)
        sig = green_sigma_hat(C, XI, eh, k0_mode, zero)
        Q[ix] = ddot6(E6[:, None, None], to_voigt6(sig).real)
    return np.fft.ifftn(Q).real


def self_term_table_realspace(d, n, h, K, s):
    """The table of ``self_term_table`` as a double sum over the two stencils in real
    space (convolution theorem applied to self_term_table_fourier): with K the kernel of
    the defect's unit tensor (e = s E) and w_c the class-c counts placed at the origin,
      W(c, 0)     = -kappa h^3 a_c^2 s^2   sum_{v,v'} w_c(v) w_c(v')  K(v' - v)
      W(c, 1 + j) = -kappa h^3 a_c a_c' s^2 sum_{v,v'} w_c(v) w_c'(v') K(v' + d_cj - v)
    with c' = 1 - c and d_cj the whole-voxel shift between the two stencils."""
    n = np.array([int(v) for v in n])
    st = [stencil(d, c, h) for c in (0, 1)]
    pref = -KAPPA * h ** 3 * s * s

    def pair_sum(c, cp, shift):
        oc, wc, _ = st[c]
        op, wp, _ = st[cp]
        tot = 0.0
        for r0 in range(0, len(oc), 256):          # rows in chunks keep the index arrays small
            r = np.mod(op[None, :, :] + shift[None, None, :] - oc[r0:r0 + 256, None, :], n)
            tot += float(np.sum(wc[r0:r0 + 256, None] * wp[None, :] * K[r[..., 0], r[..., 1], r[..., 2]]))
        return tot

    W = np.zeros((2, 9))
    for c in (0, 1):
        cp = 1 - c
        W[c, 0] = pref * st[c][2] ** 2 * pair_sum(c, c, np.zeros(3, dtype=np.int64))
        ref = np.array([c, c, c], dtype=np.int64)
        for j in range(8):
            dvec = base_voxel(ref + JUMPS[j]) - base_voxel(ref)
            W[c, 1 + j] = pref * st[c][2] * st[cp][2] * pair_sum(c, cp, dvec)
    return W


def energies_sampled(defects, sample, sigma_total, n, h, C, k0_mode=MEAN_STRESS_ZERO):
    """E_i(X_i) and E_i(X_i + lambda_j) for the sampled defects by the sigma - W route
    (Sec. 2, Eq. interaction_energy3): the stencil sum over the total stress minus the
    self term, with W from self_term_table_realspace and one kernel per unit tensor.
    Returns {i: (e0, ec[8])}."""
    kernels = {}
    out = {}
    for i in sample:
        d = defects[i]
        E, s = unit_tensor(d, h)
        key = tuple(np.round(E.ravel(), 12))
        if key not in kernels:
            kernels[key] = unit_kernel(E, n, h, C, k0_mode)
        W = self_term_table_realspace(d, n, h, kernels[key], s)
        c = pos_class(d['pos'])
        e0 = energy_of_stencil(d, d['pos'], sigma_total, h) - W[c, 0]
        ec = np.array([energy_of_stencil(d, Y, sigma_total, h) - W[c, 1 + j]
                       for j, Y in enumerate(candidate_positions(d['pos']))])
        out[int(i)] = (e0, ec)
    return out


# --------------------------------------------------------------------------
# rates and event selection (Sec. 5; Appendix A, Algorithm 1)
# --------------------------------------------------------------------------
def nominal_frequency(Em, T, nu0=NU0_DEFAULT):
    """Eq. unbiased_boltzmann."""
    return nu0 * math.exp(-Em / (KB * T))


def jump_rates(Em, E0, Ec, allowed, T, nu0=NU0_DEFAULT):
    """Biased frequencies of the allowed jumps (Eqs. biased_forward/backward_boltzmann
    with prefactor 1/z, z = number of allowed jumps); zero for the others."""
    z = int(np.sum(allowed))
    r = np.zeros(8)
    if z == 0:
        return r
    for j in range(8):
        if allowed[j]:
            r[j] = (nu0 / z) * math.exp(-(Em + 0.5 * (Ec[j] - E0)) / (KB * T))
    return r


def select_on_line(rates, u):
    """First index k with R_{k-1} < u R_tot <= R_k on the running sum (Eq. selection_jump)."""
    R = np.cumsum(rates)
    target = u * R[-1]
    k = int(np.searchsorted(R, target, side='left'))
    return min(k, len(rates) - 1), R


# ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), from its published definition
_M0, _M1 = 0xD2511F53, 0xCD9E8D57
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
_MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    x = [int(v) & _MASK for v in ctr]
    k0, k1 = int(key[0]) & _MASK, int(key[1]) & _MASK
    for r in range(10):
        if r:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * x[0]
        p1 = _M1 * x[2]
        hi0, lo0 = p0 >> 32, p0 & _MASK
        hi1, lo1 = p1 >> 32, p1 & _MASK
        x = [hi1 ^ x[1] ^ k0, lo1, hi0 ^ x[3] ^ k1, lo0]
    return x


def u53(lo, hi):
    """Uniform on (0, 1] from 53 bits: ((hi << 21) | (lo >> 11)) + 1 over 2^53."""
    return float(((hi << 21) | (lo >> 11)) + 1) * (2.0 ** -53)


def uniforms(seed, ctr):
    """Two uniforms from one Philox block; key = seed (64 bit), counter = ctr (4 words)."""
    x = philox4x32_10(ctr, (seed & _MASK, (seed >> 32) & _MASK))
    return u53(x[0], x[1]), u53(x[2], x[3])


TAG_RESIDENCE, TAG_FIXED_DT = 0, 1
NO_DEFECT = 0xFFFFFFFF


def residence_uniforms(seed, step):
    return uniforms(seed, (step & _MASK, (step >> 32) & _MASK, NO_DEFECT, TAG_RESIDENCE))


def fixed_dt_uniforms(seed, step, i):
    return uniforms(seed, (step & _MASK, (step >> 32) & _MASK, i, TAG_FIXED_DT))


def residence_step(defects, E, Ec, T, seed, step, n, nu0=NU0_DEFAULT):
    """One residence-time event: every allowed jump of every defect on one frequency
    line; returns (i, j, dt, R_tot) and moves defect i in place."""
    rates = np.concatenate([jump_rates(float(d['Em_eV']), E[i], Ec[i], allowed_jumps(d), T, nu0)
                            for i, d in enumerate(defects)])
    u1, u2 = residence_uniforms(seed, step)
    k, R = select_on_line(rates, u1)
    i, j = divmod(k, 8)
    dt = -math.log(u2) / R[-1]
    p = np.mod(np.asarray(defects[i]['pos'], dtype=np.int64) + JUMPS[j], 2 * np.asarray(n))
    defects[i]['pos'] = p
    return i, j, dt, R[-1]


def fixed_dt(defects, T, nu0=NU0_DEFAULT):
    """delta t = 1/nu_max over the mobile defects, nominal barriers (Eq. time_step)."""
    nus = [nominal_frequency(float(d['Em_eV']), T, nu0) for d in defects
           if int(d['mobility']) != IMMOBILE]
    return 1.0 / max(nus)


def fixed_dt_step(defects, E, Ec, T, seed, step, n, dt, nu0=NU0_DEFAULT):
    """One synchronous step of Algorithm 1: each mobile defect draws its Poisson count
    with the nominal frequency; if it is > 0 it selects one jump on its biased
    frequency line.  All decisions use the start-of-step energies; moves are applied
    together.  Returns the list of (i, j) jumps."""
    moves = []
    for i, d in enumerate(defects):
        al = allowed_jumps(d)
        if not al.any():
            continue
        up, us = fixed_dt_uniforms(seed, step, i)
        mu = nominal_frequency(float(d['Em_eV']), T, nu0) * dt
        if up <= math.exp(-mu):             # N_i = 0 by CDF inversion (Eq. poisson)
            continue
        r = jump_rates(float(d['Em_eV']), E[i], Ec[i], al, T, nu0)
        j, _ = select_on_line(r, us)
        moves.append((i, j))
    for i, j in moves:
        defects[i]['pos'] = np.mod(np.asarray(defects[i]['pos'], dtype=np.int64) + JUMPS[j],
                                   2 * np.asarray(n))
    return moves


# --------------------------------------------------------------------------
# the paper's translation of a defect's field by the shift theorem (Sec. 3.3, Eq. shift):
# the elastic strain spectrum of the defect at a reference site is stored once and
# moved to any (continuous) position X by exp(-i xi.(X - X0)); the energy is the paper
# form of Eq. interaction_energy3, kappa int sigma_ext : eps^{d,e}(X) dV
# --------------------------------------------------------------------------
def elastic_strain_spectrum(d, n, h, C, k0_mode=MEAN_STRESS_ZERO):
    """(X0 in nm, eps_hat (6, nx, ny, nz)): the defect alone at the class-0 reference site
    pos = 0 (centre at the origin corner), its elastic strain C^-1 : sigma_d (engineering
    shears halved to tensor components) and that field's transform."""
    dd = as_record(d)
    dd['pos'] = np.zeros(3, dtype=np.int64)
    sig = solve_stress(eigenstrain_field([dd], n, h), C, h, k0_mode)
    S = np.linalg.inv(stiffness_matrix(C))
    eps = np.einsum('ab,b...->a...', S, sig)
    eps[3:] *= 0.5
    return np.zeros(3), np.fft.fftn(eps, axes=(-3, -2, -1))


def shifted_field(eps_hat, shift, h):
    """The field of eps_hat moved by `shift` (nm): Re ifft(exp(-i xi.shift) eps_hat)."""
    n = eps_hat.shape[1:]
    xs = [frequencies(n[a], n[a] * h) for a in range(3)]
    ph = np.exp(-1j * (xs[0][:, None, None] * shift[0] + xs[1][None, :, None] * shift[1]
                       + xs[2][None, None, :] * shift[2]))
    return np.fft.ifftn(eps_hat * ph[None], axes=(-3, -2, -1)).real


def energy_shift_theorem(eps_ref, X, sigma_ext, h):
    """kappa int sigma_ext : eps^{d,e}(X) dV with the defect's elastic strain moved from
    the reference site to X (nm) by Eq. shift, summed by Parseval:
      (h^3 / N) Re sum_xi conj(sigma_ext_hat) : eps_hat exp(-i xi.(X - X0))."""
    X0, eps_hat = eps_ref
    n = sigma_ext.shape[1:]
    xs = [frequencies(n[a], n[a] * h) for a in range(3)]
    dX = np.asarray(X, float) - X0
    ph = np.exp(-1j * (xs[0][:, None, None] * dX[0] + xs[1][None, :, None] * dX[1]
                       + xs[2][None, None, :] * dX[2]))
    sh = np.fft.fftn(sigma_ext, axes=(-3, -2, -1))
    return KAPPA * h ** 3 / np.prod(n) * float(np.sum(ddot6(np.conj(sh), eps_hat * ph[None])).real)


# --------------------------------------------------------------------------
# dislocation lines by field dislocation mechanics (Sec. 3.2: Eqs. Nye2, curlUe,
# eq_EIG_fourier, plastic_0); voxel centres at (v + 1/2) h (Sec. 3.4)
# --------------------------------------------------------------------------
LEVI_CIVITA = np.zeros((3, 3, 3))
for _i, _j, _k in ((0, 1, 2), (1, 2, 0), (2, 0, 1)):
    LEVI_CIVITA[_i, _j, _k] = 1.0
    LEVI_CIVITA[_i, _k, _j] = -1.0


def nye_tensor(points, b, n, h, closed=True, ds_max=None):
    """Nye tensor alpha_ij (3, 3, nx, ny, nz) of a polyline dislocation with Burgers
    vector b (nm): Eq. Nye2, the Burgers vector density of each sub-segment (length at
    most ds_max, default h/4) spread to the 8 voxel centres around its midpoint with
    trilinear weights (the paper spreads the core over the 8 surrounding grid points,
    Sec. 4).  alpha_ij(v) = sum_s b_i t_j ds w_s(v) / h^3.  An open polyline whose end
    is a lattice translate of its start is a periodic (infinite) line."""
    n = tuple(int(v) for v in n)
    ds_max = ds_max or 0.25 * h
    P = np.asarray(points, dtype=np.float64)
    ends = list(zip(P[:-1], P[1:])) + ([(P[-1], P[0])] if closed else [])
    xs, ts, dss = [], [], []
    for p, q in ends:
        d = q - p
        L = float(np.linalg.norm(d))
        m = max(1, int(math.ceil(L / ds_max)))
        t = d / L
        k = (np.arange(m) + 0.5)[:, None]
        xs.append(p[None, :] + k * (L / m) * t[None, :])
        ts.append(np.repeat(t[None, :], m, axis=0))
        dss.append(np.full(m, L / m))
    X, T, DS = np.concatenate(xs), np.concatenate(ts), np.concatenate(dss)
    u = X / h - 0.5
    i0 = np.floor(u).astype(np.int64)
    f = u - i0
    alpha = np.zeros((3, 3) + n)
    bt = np.einsum('i,sj->sij', np.asarray(b, float), T) * (DS / h ** 3)[:, None, None]
    for cx in (0, 1):
        for cy in (0, 1):
            for cz in (0, 1):
                w = ((f[:, 0] if cx else 1 - f[:, 0]) * (f[:, 1] if cy else 1 - f[:, 1])
                     * (f[:, 2] if cz else 1 - f[:, 2]))
                idx = np.mod(i0 + np.array([cx, cy, cz])[None, :], np.array(n)[None, :])
                for i in range(3):
                    for j in range(3):
                        np.add.at(alpha[i, j], (idx[:, 0], idx[:, 1], idx[:, 2]), w * bt[:, i, j])
    return alpha


def plastic_distortion(alpha, h, U0=None):
    """U^p (3, 3, nx, ny, nz): the incompatible part of Eq. eq_EIG_fourier,
    U_hat_ij = -i xi_k / |xi|^2 eps_jkl alpha_hat_il for xi != 0, plus a uniform
    compatible part U0 (3x3) as the xi = 0 term (Eq. plastic_0); the real part of the
    inverse transform (the even-edge Nyquist reading of the stress solve)."""
    n = alpha.shape[2:]
    xs = [frequencies(n[a], n[a] * h) for a in range(3)]
    XI = np.stack(np.meshgrid(xs[0], xs[1], xs[2], indexing='ij'))          # (3, nx, ny, nz)
    xi2 = np.sum(XI * XI, axis=0)
    zero = xi2 == 0.0
    q = XI / np.where(zero, 1.0, xi2)[None]
    ah = np.fft.fftn(alpha, axes=(-3, -2, -1))
    Uh = -1j * np.einsum('kxyz,jkl,ilxyz->ijxyz', q, LEVI_CIVITA, ah)
    Uh[:, :, zero] = 0.0
    if U0 is not None:
        Uh[:, :, zero] = (np.asarray(U0, float) * np.prod(n))[:, :, None]
    return np.fft.ifftn(Uh, axes=(-3, -2, -1)).real


def dislocation_eigenstrain6(alpha, h, U0=None):
    """eps_EIG = sym(U^p), 6 components (the plastic strain taken as eigenstrain)."""
    U = plastic_distortion(alpha, h, U0)
    return to_voigt6(0.5 * (U + np.transpose(U, (1, 0, 2, 3, 4))))


def circle_points(center, normal, R, m=256):
    """m points of the circle of radius R about `normal` (unit), counter-clockwise seen
    from the normal's tip, so that its oriented area is pi R^2 normal."""
    nv = np.asarray(normal, float) / np.linalg.norm(normal)
    a = np.array([1.0, 0.0, 0.0]) if abs(nv[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(nv, a)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(nv, e1)
    th = 2.0 * PI * np.arange(m) / m
    return np.asarray(center, float)[None, :] + R * (np.cos(th)[:, None] * e1[None, :] + np.sin(th)[:, None] * e2[None, :])


# --------------------------------------------------------------------------
# dipole approximation of the interaction energy (Sec. 2.1, Eqs. interaction_energy4,
# dipole_def, dipole_def2; Appendix B): with the external field taken constant over the
# defect, E_i(Y) ~ -P_i : eps_ext(Y) = -(int eps*_i) : sigma^(-i)(Y), since
# P_i = C : int eps*_i and sigma^(-i) = C : eps_ext where the other defects' eigenstrain
# vanishes.
# --------------------------------------------------------------------------
def integrated_eigenstrain6(d, h):
    """int eps*_d dV (6 components, nm^3): the shape volume times e (P = C : this)."""
    g = defect_geometry(d, h)
    return g['v_over_h3'] * h ** 3 * to_voigt6(g['e'])


def center_voxels(pos):
    """Voxels whose mean is a field's value at the centre of a defect at pos.  With the
    subsample coordinates of ``stencil``, a class-1 centre is the centre of its base
    voxel, and a class-0 centre the corner shared by the 8 voxels base + {-1, 0}^3
    (trilinear interpolation of voxel-centred values there is their mean)."""
    b = base_voxel(pos)
    if pos_class(pos) == 1:
        return b[None, :]
    return b[None, :] + np.array([[i, j, k] for i in (-1, 0) for j in (-1, 0) for k in (-1, 0)],
                                 dtype=np.int64)


def sample_center(field6, pos):
    """field6 (6, nx, ny, nz) at the centre of a defect at half-lattice position pos."""
    n = np.array(field6.shape[1:])
    v = np.mod(center_voxels(pos), n[None, :])
    return field6[:, v[:, 0], v[:, 1], v[:, 2]].mean(axis=1)


def dipole_energy_at(d, pos_Y, sigma6, h):
    """-kappa (int eps*_d) : sigma(Y) for defect d with its centre at pos_Y."""
    return -KAPPA * ddot6(integrated_eigenstrain6(d, h), sample_center(sigma6, pos_Y))


# Table 1: dipole tensor of the <110> dumbbell self-interstitial in Fe (eV), printed as
# P11, P22, P33, P12, P13, P23; here in VOIGT order (xx, yy, zz, yz, xz, xy).
SIA_110_DIPOLE_EV = np.array([25.832, 21.143, 21.150, 5.122, 0.000, 0.000])


def point_dipole_energy(P6, pos_Y, sigma6, C):
    """E = -P : eps(Y) (Eq. interaction_energy4) for a point defect of dipole tensor P
    (eV; VOIGT order) with its centre at site pos_Y: eps = C^-1 : sigma read at the
    centre of the site (``sample_center``).  With engineering shear strains, P : eps is
    the plain sum of the six products."""
    e = np.linalg.solve(stiffness_matrix(C), sample_center(sigma6, pos_Y))
    return -float(np.dot(np.asarray(P6, float), e))


def dipole_energies(defects, n, h, C, k0_mode=MEAN_STRESS_ZERO):
    """Dipole-approximation energies of every defect at its site and at its eight jumps,
    with sigma^(-i) = sigma - sigma_i (sigma_i from the solve of defect i alone)."""
    sig = solve_stress(eigenstrain_field(defects, n, h), C, h, k0_mode)
    E = np.zeros(len(defects))
    Ec = np.zeros((len(defects), 8))
    for i, d in enumerate(defects):
        s = sig - solve_stress(eigenstrain_field(defects, n, h, only={i}), C, h, k0_mode)
        E[i] = dipole_energy_at(d, d['pos'], s, h)
        for j, Y in enumerate(candidate_positions(d['pos'])):
            Ec[i, j] = dipole_energy_at(d, Y, s, h)
    return E, Ec


def dipole_self_table(d, n, h, C, k0_mode=MEAN_STRESS_ZERO):
    """D(c, k) = (int eps*_d) : sigma_d(Y_k) (GPa nm^3): the defect's own field at the centre
    Y_0 of a reference site of class c, or at its jump k - 1, contracted with its
    integrated eigenstrain.  Kappa times it is the self part that sigma^(-i) removes
    from a dipole energy.  Translation invariant under whole-voxel shifts, like
    ``self_term_table``."""
    D = np.zeros((2, 9))
    ie = integrated_eigenstrain6(d, h)
    for c in (0, 1):
        ref = np.array([c, c, c], dtype=np.int64)
        dd = as_record(d)
        dd['pos'] = ref
        sig = solve_stress(eigenstrain_field([dd], n, h), C, h, k0_mode)
        D[c, 0] = ddot6(ie, sample_center(sig, ref))
        for j, Y in enumerate(candidate_positions(ref)):
            D[c, 1 + j] = ddot6(ie, sample_center(sig, Y))
    return D


def dipole_self_table_fourier(d, n, h, C, k0_mode=MEAN_STRESS_ZERO):
    """The table of ``dipole_self_table`` by Fourier sums: with w_c the count field of the
    class-c stencil placed at the origin and q(xi) = e : sigma_hat[e](xi),
      D(c, k) = V_shape a_c / N  Re sum_xi q(xi) w_c(xi) S_k(xi),
    S_k(xi) the mean of exp(+i xi.v) over the centre voxels v of Y_k (relative to the
    reference site's base voxel)."""
    n = tuple(int(v) for v in n)
    N = n[0] * n[1] * n[2]
    g = defect_geometry(d, h)
    e = g['e']
    e6 = to_voigt6(e)
    V = g['v_over_h3'] * h ** 3
    xs = [frequencies(n[a], n[a] * h) for a in range(3)]
    fr = [np.fft.fftfreq(n[a]) * n[a] for a in range(3)]
    q = np.empty(n)
    for ix in range(n[0]):
        XI = np.stack(np.meshgrid(np.full(1, xs[0][ix]), xs[1], xs[2], indexing='ij'), axis=-1)[0]
        zero = np.all(XI == 0.0, axis=-1)
        eh = np.broadcast_to(e[:, :, None, None], (3, 3) + XI.shape[:2]).astype(complex)
        sig = green_sigma_hat(C, XI, eh, k0_mode, zero)
        q[ix] = ddot6(e6[:, None, None], to_voigt6(sig).real)
    D = np.zeros((2, 9))
    for c in (0, 1):
        offs, cnt, a = stencil(d, c, h)
        f = np.zeros(n)
        v = np.mod(offs, np.array(n)[None, :])
        np.add.at(f, (v[:, 0], v[:, 1], v[:, 2]), cnt.astype(float))
        what = np.fft.fftn(f)
        ref = np.array([c, c, c], dtype=np.int64)
        for k, Y in enumerate([ref] + candidate_positions(ref)):
            S = np.zeros(n, dtype=complex)
            for vv in center_voxels(Y) - base_voxel(ref)[None, :]:
                S += np.exp(2j * PI * (fr[0][:, None, None] * vv[0] / n[0] + fr[1][None, :, None] * vv[1] / n[1]
                                       + fr[2][None, None, :] * vv[2] / n[2]))
            S /= len(center_voxels(Y))
            D[c, k] = V * a / N * np.sum(q * what * S).real
    return D


# --------------------------------------------------------------------------
# dipole-limit helpers for the far-field pin (Sec. 2.1, Eqs. interaction_energy4, dipole_DL)
# --------------------------------------------------------------------------
def loop_dipole_tensor(C, b, A):
    """P = (1/2) C : (b (x) A + A (x) b) (Eq. dipole_DL)."""
    S = 0.5 * (np.outer(b, A) + np.outer(A, b))
    return np.einsum('ijkl,kl->ij', C, S)


def blin_interaction_energy(line1, b1, line2, b2, mu, nu):
    """Interaction energy (GPa nm^3) of two closed dislocation lines in an infinite
    isotropic body, by Blin's double line integral (Hirth & Lothe, Theory of
    Dislocations, Ch. 4):
      W = -mu/(2 pi) oint oint (b1 x b2).(dl1 x dl2)/R + mu/(4 pi) oint oint (b1.dl1)(b2.dl2)/R
          + mu/(4 pi (1 - nu)) oint oint (b1 x dl1).T.(b2 x dl2),   T_ij = d_i d_j R,
    R = |x2 - x1|, evaluated by the midpoint rule over the polylines' segments (the lines
    must not touch).  T_ij = (delta_ij - u_i u_j)/R with u the unit vector along x2 - x1.
    Bilinear in (b, dl) of each line, so the result does not depend on the line-sense
    convention as long as both lines follow the same one."""
    P1, P2 = np.asarray(line1, float), np.asarray(line2, float)
    d1 = np.roll(P1, -1, axis=0) - P1
    d2 = np.roll(P2, -1, axis=0) - P2
    Rv = (P2 + 0.5 * d2)[None, :, :] - (P1 + 0.5 * d1)[:, None, :]
    R = np.linalg.norm(Rv, axis=2)
    u = Rv / R[..., None]
    b1, b2 = np.asarray(b1, float), np.asarray(b2, float)
    t1 = np.einsum('k,abk->ab', np.cross(b1, b2), np.cross(d1[:, None, :], d2[None, :, :])) / R
    t2 = np.outer(d1 @ b1, d2 @ b2) / R
    c1, c2 = np.cross(b1, d1), np.cross(b2, d2)
    t3 = (c1 @ c2.T - np.einsum('ai,abi->ab', c1, u) * np.einsum('bi,abi->ab', c2, u)) / R
    return (-mu / (2.0 * PI) * t1.sum() + mu / (4.0 * PI) * t2.sum()
            + mu / (4.0 * PI * (1.0 - nu)) * t3.sum())


def kelvin_green(x, mu, nu):
    """Isotropic infinite-body Green's function G_ik(x) (Kelvin solution)."""
    r = np.linalg.norm(x)
    return ((3.0 - 4.0 * nu) * np.eye(3) + np.outer(x, x) / r ** 2) / (16.0 * PI * mu * (1.0 - nu) * r)


def dipole_dipole_energy(P1, P2, d, mu, nu, step=1e-3):
    """E = P1_ij P2_kl d_j d_l G_ik(d), second derivatives by central differences."""
    s = step * np.linalg.norm(d)
    D = np.zeros((3, 3, 3, 3))       # D[i,k,j,l] = d_j d_l G_ik
    I = np.eye(3)
    for j in range(3):
        for l in range(3):
            g = (kelvin_green(d + s * I[j] + s * I[l], mu, nu)
                 - kelvin_green(d + s * I[j] - s * I[l], mu, nu)
                 - kelvin_green(d - s * I[j] + s * I[l], mu, nu)
                 + kelvin_green(d - s * I[j] - s * I[l], mu, nu)) / (4.0 * s * s)
            D[:, :, j, l] = g
    return float(np.einsum('ij,kl,ikjl->', P1, P2, D))
