"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a naive DFT,
closed forms, invariants, the paper's printed numbers (tests/golden/), brute
force on tiny grids, or a statistical law.  No GPU needed.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2403_09158_gb300.workload import DEFECT_DTYPE, make_defects

GOLD = os.path.join(os.path.dirname(__file__), 'golden')
H = 0.2855
C_CUBIC = O.stiffness_cubic(243.0, 145.0, 116.0)


def _defects_small(n=16):
    """A loop, a <100> loop and two SIA clusters inside a small box."""
    return make_defects(
        [O.LOOP_111, O.LOOP_100, O.SIA_CLUSTER, O.SIA_CLUSTER],
        np.array([[4, 4, 4], [19, 13, 21], [10, 26, 6], [27, 7, 15]]),
        [1, 2, 0, 3], [0.55, 0.5, 0.0, 0.0], [0, 0, 3, 1], [0.1, 1.0, 0.3, 0.3],
        [O.ONE_D, O.IMMOBILE, O.ONE_D, O.THREE_D])


# ---------------------------------------------------------------- P1: transforms
@pytest.mark.parametrize('n', [(6, 10, 15), (8, 12, 5), (16, 6, 9)])
def test_p1_solve_with_naive_dft_matches(n):
    rng = np.random.default_rng(1)
    eps = rng.normal(size=(6,) + n)
    a = O.solve_stress(eps, C_CUBIC, H, O.MEAN_STRESS_ZERO)
    b = O.solve_stress(eps, C_CUBIC, H, O.MEAN_STRESS_ZERO, dft=O.naive_dft_pair(n))
    assert np.linalg.norm(a - b) <= 1e-12 * np.linalg.norm(a)
    fwd, _ = O.naive_dft_pair(n)
    x = rng.normal(size=n)
    assert np.allclose(fwd(x), np.fft.fftn(x), rtol=0, atol=1e-10)


def test_p1_frequencies_follow_paper_convention():
    # Eq. frequencies: n = m - N/2 (even N) after centring: the set {-N/2 .. N/2-1}
    f = O.frequencies(8, 8.0) * 8.0 / (2 * np.pi)
    assert sorted(np.round(f).astype(int).tolist()) == list(range(-4, 4))
    f = O.frequencies(7, 7.0) * 7.0 / (2 * np.pi)
    assert sorted(np.round(f).astype(int).tolist()) == list(range(-3, 4))


# ---------------------------------------------------------------- P2: uniform eigenstrain
@pytest.mark.parametrize('n', [(8, 8, 8), (6, 10, 5)])
def test_p2_uniform_eigenstrain(n):
    e6 = np.array([1e-3, -2e-3, 5e-4, 3e-4, -1e-4, 2e-4])
    eps = np.broadcast_to(e6[:, None, None, None], (6,) + n).copy()
    s0 = O.solve_stress(eps, C_CUBIC, H, O.MEAN_STRESS_ZERO)
    assert np.abs(s0).max() < 1e-13
    s1 = O.solve_stress(eps, C_CUBIC, H, O.MEAN_STRAIN_ZERO)
    expect = -O.to_voigt6(np.einsum('ijkl,kl->ij', C_CUBIC, O.to_tensor(e6)))
    assert np.abs(s1 - expect[:, None, None, None]).max() < 1e-13


# ---------------------------------------------------------------- P3: per-frequency identities
def test_p3_idempotence_equilibrium_compatibility():
    rng = np.random.default_rng(2)
    C9 = C_CUBIC.reshape(9, 9)
    for _ in range(20):
        xi = rng.normal(size=3)
        G = O.green_operator_matrix(C_CUBIC, xi)
        G9 = G.reshape(9, 9)
        assert np.abs(G9 @ C9 @ G9 - G9).max() < 1e-13 * np.abs(G9).max() * 50
        # sigma_hat = C:(Gamma:tau - eps*) must satisfy m . sigma_hat = 0 (equilibrium)
        tau = O.to_tensor(rng.normal(size=6))
        eps_star = O.strain_from_engineering(np.linalg.solve(O.stiffness_matrix(C_CUBIC), O.stress_vec(tau)))
        sig = O.green_sigma_hat(C_CUBIC, xi[None, :], eps_star[:, :, None].astype(complex),
                                O.MEAN_STRESS_ZERO, np.zeros(1, bool))[:, :, 0]
        m = xi / np.linalg.norm(xi)
        assert np.abs(sig @ m).max() < 1e-12 * np.abs(sig).max()
        # the total strain Gamma:tau is compatible: P_perp eps P_perp = 0
        eps = np.einsum('ijkl,kl->ij', G, tau)
        P = np.eye(3) - np.outer(m, m)
        assert np.abs(P @ eps @ P).max() < 1e-13 * np.abs(eps).max() * 10


def test_p3_real_space_equilibrium_on_odd_grid():
    # odd edges have no Nyquist index, so discrete equilibrium holds at every frequency
    n = (9, 7, 11)
    rng = np.random.default_rng(3)
    sig = O.solve_stress(rng.normal(size=(6,) + n), C_CUBIC, H, O.MEAN_STRESS_ZERO)
    sh = O.to_tensor(np.fft.fftn(sig, axes=(1, 2, 3)))
    xs = [O.frequencies(n[a], n[a] * H) for a in range(3)]
    XI = np.stack(np.meshgrid(*xs, indexing='ij'), axis=0)
    div = np.einsum('ij...,j...->i...', sh, XI)
    assert np.abs(div).max() < 1e-11 * np.abs(sh).max()


# ---------------------------------------------------------------- P4: isotropic closed form
def test_p4_isotropic_matches_moulinec_suquet():
    mu, nu = 82.0, 0.29
    C11, C12, C44 = O.isotropic_cubic_constants(mu, nu)
    lam = C12
    C = O.stiffness_cubic(C11, C12, C44)
    d = np.eye(3)
    rng = np.random.default_rng(4)
    for _ in range(10):
        xi = rng.normal(size=3)
        x2 = xi @ xi
        ref = (np.einsum('ki,h,j->khij', d, xi, xi) + np.einsum('hi,k,j->khij', d, xi, xi)
               + np.einsum('kj,h,i->khij', d, xi, xi) + np.einsum('hj,k,i->khij', d, xi, xi)) / (4 * mu * x2)
        ref -= (lam + mu) / (mu * (lam + 2 * mu)) * np.einsum('i,j,k,h->khij', xi, xi, xi, xi) / x2 ** 2
        G = O.green_operator_matrix(C, xi)
        assert np.abs(G - ref).max() < 1e-14 * 1e3 * np.abs(ref).max()


# ---------------------------------------------------------------- P5/P6: energies
def test_p5_reciprocity():
    n = (16, 16, 16)
    d = _defects_small()
    i, j = 0, 2
    s_j = O.solve_stress(O.eigenstrain_field(d, n, H, only={j}), C_CUBIC, H)
    s_i = O.solve_stress(O.eigenstrain_field(d, n, H, only={i}), C_CUBIC, H)
    Eij = O.energy_of_stencil(d[i], d[i]['pos'], s_j, H)
    Eji = O.energy_of_stencil(d[j], d[j]['pos'], s_i, H)
    assert abs(Eij) > 1e-4
    assert abs(Eij - Eji) <= 1e-10 * abs(Eij)


def test_p6_bruteforce_equals_self_field_and_table():
    n = (16, 16, 16)
    d = _defects_small()
    E, Ec = O.energies_bruteforce(d, n, H, C_CUBIC)
    res, sig = O.energies_self_field(d, n, H, C_CUBIC)
    for i in range(len(d)):
        assert abs(res[i][0] - E[i]) <= 1e-10 * max(1.0, abs(E[i]))
        assert np.abs(res[i][1] - Ec[i]).max() <= 1e-10 * max(1.0, np.abs(Ec[i]).max())
        # table route: total-field energy minus the translation-invariant self term
        W = O.self_term_table(d[i], n, H, C_CUBIC)
        Wf = O.self_term_table_fourier(d[i], n, H, C_CUBIC)
        assert np.abs(W - Wf).max() <= 1e-10 * np.abs(W).max()
        c = O.pos_class(d[i]['pos'])
        e0 = O.energy_of_stencil(d[i], d[i]['pos'], sig, H) - W[c, 0]
        assert abs(e0 - E[i]) <= 1e-9 * max(1.0, np.abs(W).max())
        for jj, Y in enumerate(O.candidate_positions(d[i]['pos'])):
            ej = O.energy_of_stencil(d[i], Y, sig, H) - W[c, 1 + jj]
            assert abs(ej - Ec[i, jj]) <= 1e-9 * max(1.0, np.abs(W).max())


@pytest.mark.parametrize('n,k0', [((16, 16, 16), O.MEAN_STRESS_ZERO), ((12, 16, 20), O.MEAN_STRAIN_ZERO)])
def test_p6_realspace_self_terms_equal_bruteforce(n, k0):
    """The sampled-energy route used at full sizes (self terms as real-space double sums
    over one kernel per unit tensor) against brute force (N_d + 1 solves)."""
    d = _defects_small()
    E, Ec = O.energies_bruteforce(d, n, H, C_CUBIC, k0)
    sig = O.solve_stress(O.eigenstrain_field(d, n, H), C_CUBIC, H, k0)
    res = O.energies_sampled(d, range(len(d)), sig, n, H, C_CUBIC, k0)
    for i in range(len(d)):
        W = O.self_term_table_fourier(d[i], n, H, C_CUBIC, k0)
        E_, s = O.unit_tensor(d[i], H)
        assert abs(s * E_ - O.defect_geometry(d[i], H)['e']).max() <= 1e-15
        Wr = O.self_term_table_realspace(d[i], n, H, O.unit_kernel(E_, n, H, C_CUBIC, k0), s)
        assert np.abs(Wr - W).max() <= 1e-12 * np.abs(W).max()
        assert abs(res[i][0] - E[i]) <= 1e-9 * max(1.0, np.abs(W).max())
        assert np.abs(res[i][1] - Ec[i]).max() <= 1e-9 * max(1.0, np.abs(W).max())


def test_p6_paper_form_equals_eigenstrain_form():
    # Eq. interaction_energy3: int sigma_ext : eps^{d,e} = -int sigma_ext : eps*_d.  Exact on
    # odd edges; on even edges the averaged Nyquist operator breaks it by a few 1e-3.
    n = (15, 15, 15)
    d = _defects_small()
    i = 1
    s_ext = O.solve_stress(O.eigenstrain_field(d, n, H, exclude={i}), C_CUBIC, H)
    eps_i = O.eigenstrain_field(d, n, H, only={i})
    s_i = O.solve_stress(eps_i, C_CUBIC, H)
    S = np.linalg.inv(O.stiffness_matrix(C_CUBIC))
    # elastic strain of defect i alone, eps^{d,e} = C^-1 : sigma_i (engineering -> tensor)
    eng = np.einsum('ab,b...->a...', S, s_i)
    eps_e = eng.copy()
    eps_e[3:] *= 0.5
    lhs = O.KAPPA * H ** 3 * np.sum(O.ddot6(s_ext, eps_e))
    rhs = -O.KAPPA * H ** 3 * np.sum(O.ddot6(s_ext, eps_i))
    assert abs(lhs - rhs) <= 1e-10 * abs(rhs)


# ---------------------------------------------------------------- P7: zero-frequency modes
def test_p7_k0_modes():
    n = (16, 16, 16)
    d = _defects_small()
    E0, Ec0 = O.energies_bruteforce(d, n, H, C_CUBIC, O.MEAN_STRESS_ZERO)
    E1, Ec1 = O.energies_bruteforce(d, n, H, C_CUBIC, O.MEAN_STRAIN_ZERO)
    dE0 = Ec0 - E0[:, None]
    dE1 = Ec1 - E1[:, None]
    assert np.abs(dE0 - dE1).max() < 1e-10
    Vtot = np.prod(n) * H ** 3
    for i in range(len(d)):
        e_others = O.eigenstrain_field(d, n, H, exclude={i}).reshape(6, -1).mean(axis=1)
        sbar = -O.to_voigt6(np.einsum('ijkl,kl->ij', C_CUBIC, O.to_tensor(e_others)))
        int_eps_i = O.eigenstrain_field(d, n, H, only={i}).reshape(6, -1).sum(axis=1) * H ** 3
        shift = -O.KAPPA * O.ddot6(int_eps_i, sbar)
        assert abs((E1[i] - E0[i]) - shift) < 1e-10 * max(1.0, abs(shift))
    assert Vtot > 0


# ---------------------------------------------------------------- P8: dipole far field
def test_p8_dipole_limit_isotropic():
    """Far field (Sec. 2.1, Eq. interaction_energy4 with P from Appendix B): the energy
    change between separations along a ray tends to the Kelvin dipole-dipole value as
    (R/d)^2 -> 0, and the periodic solution differs from the infinite body by a constant
    (the box's mean field) that scales as 1/V."""
    mu, nu = 82.0, 0.29
    C = O.stiffness_cubic(*O.isotropic_cubic_constants(mu, nu))
    offsets = {}
    for N in (64, 96):
        n = (N, N, N)
        c0 = np.array([N, N, N])
        loop = dict(type=O.LOOP_111, pos=c0, axis=0, radius_nm=0.35, size=0, Em_eV=0.1,
                    mobility=O.ONE_D)
        eps = O.eigenstrain_field([loop], n, H)
        s0 = O.solve_stress(eps, C, H, O.MEAN_STRAIN_ZERO)
        P = np.einsum('ijkl,kl->ij', C, O.to_tensor(eps.reshape(6, -1).sum(axis=1) * H ** 3))
        rows = []
        for step in (6, 8, 10, 12, 14):
            p2 = c0 + step * np.array([2, 1, -1])
            E = O.energy_of_stencil(dict(loop, pos=p2), p2, s0, H)
            Ed = O.dipole_dipole_energy(P, P, (p2 - c0) * H / 2.0, mu, nu) * O.KAPPA
            rows.append((E, Ed))
        offsets[N] = rows[3][0] - rows[3][1]
        if N == 96:
            errs = [abs((rows[k + 1][0] - rows[k][0]) / (rows[k + 1][1] - rows[k][1]) - 1.0)
                    for k in range(len(rows) - 1)]
            assert all(errs[k + 1] < errs[k] for k in range(len(errs) - 1)), errs
            assert errs[-1] < 5e-3
    ratio = offsets[64] / offsets[96]
    assert abs(ratio / (96.0 / 64.0) ** 3 - 1.0) < 0.15, offsets


def test_p11_integrated_eigenstrain_and_dipole_identity():
    n = (16, 16, 16)
    loop = dict(type=O.LOOP_111, pos=np.array([9, 9, 9]), axis=2, radius_nm=0.7, size=0,
                Em_eV=0.1, mobility=O.ONE_D)
    eps = O.eigenstrain_field([loop], n, H)
    int_eps = eps.reshape(6, -1).sum(axis=1) * H ** 3
    g = O.defect_geometry(loop, H)
    A = np.pi * 0.7 ** 2 * g['n']
    expect = O.to_voigt6(0.5 * (np.outer(g['b'], A) + np.outer(A, g['b'])))
    assert np.abs(int_eps - expect).max() < 1e-12
    s = O.solve_stress(eps, C_CUBIC, H, O.MEAN_STRAIN_ZERO)
    P_field = -s.reshape(6, -1).sum(axis=1) * H ** 3
    P_app_b = O.to_voigt6(O.loop_dipole_tensor(C_CUBIC, g['b'], A))
    assert np.abs(P_field - P_app_b).max() < 1e-12 * np.abs(P_app_b).max()
    sia = dict(type=O.SIA_CLUSTER, pos=np.array([8, 8, 8]), axis=0, radius_nm=0.0, size=4,
               Em_eV=0.3, mobility=O.ONE_D)
    tr = O.eigenstrain_field([sia], n, H).reshape(6, -1).sum(axis=1)[:3].sum() * H ** 3
    assert abs(tr - 1.5 * 4 * H ** 3 / 2.0) < 1e-14


# ---------------------------------------------------------------- P10: translation invariance
def test_p10_shift_invariance():
    n = (16, 16, 16)
    d = _defects_small()
    E, Ec = O.energies_bruteforce(d, n, H, C_CUBIC)
    d2 = d.copy()
    d2['pos'] = np.mod(d2['pos'] + np.array([6, -4, 10]), 32)
    E2, Ec2 = O.energies_bruteforce(d2, n, H, C_CUBIC)
    assert np.abs(E2 - E).max() < 1e-12 and np.abs(Ec2 - Ec).max() < 1e-12


# ---------------------------------------------------------------- stencils
@pytest.mark.parametrize('rec', [
    dict(type=0, axis=0, radius_nm=1.3, size=0), dict(type=0, axis=3, radius_nm=0.52, size=0),
    dict(type=1, axis=1, radius_nm=0.9, size=0), dict(type=2, axis=0, radius_nm=0.0, size=1),
    dict(type=2, axis=0, radius_nm=0.0, size=40)])
def test_stencil_volume_and_real_coordinate_coverage(rec):
    rec = dict(rec, pos=np.array([0, 0, 0]), Em_eV=0.1, mobility=0)
    g = O.defect_geometry(rec, H)
    rng = np.random.default_rng(5)
    for c in (0, 1):
        offs, cnt, alpha = O.stencil(rec, c, H)
        assert abs(cnt.sum() * alpha - g['v_over_h3']) < 1e-12 * g['v_over_h3']
        # recount a few voxels from real coordinates (centre at c*(h/2) per axis)
        X = np.full(3, c * H / 2.0)
        table = {tuple(o): k for o, k in zip(offs.tolist(), cnt.tolist())}
        cand = list(table.keys())[:12] + [tuple(v) for v in rng.integers(-3, 4, (12, 3))]
        for v in cand:
            k = 0
            for i in range(4):
                for j in range(4):
                    for l in range(4):
                        x = (np.array(v) + (np.array([i, j, l]) + 0.5) / 4.0) * H - X
                        if g['kind'] == 'disk':
                            t = x @ g['n']
                            inside = abs(t) <= H / 2 + 1e-12 and (x @ x - t * t) <= g['R'] ** 2 + 1e-12
                        else:
                            inside = x @ x <= (g['v_over_h3'] * 3 / (4 * np.pi)) ** (2 / 3) * H ** 2 + 1e-12
                        k += inside
            assert k == table.get(tuple(v), 0), (c, v)


def test_stencil_point_symmetry():
    rec = dict(type=0, axis=2, radius_nm=1.1, size=0, pos=np.array([0, 0, 0]), Em_eV=0.1, mobility=0)
    o1, c1, _ = O.stencil(rec, 1, H)        # centre at a voxel centre: v -> -v
    t1 = {tuple(o): k for o, k in zip(o1.tolist(), c1.tolist())}
    assert all(t1[tuple(-np.array(o))] == k for o, k in t1.items())
    o0, c0, _ = O.stencil(rec, 0, H)        # centre at a voxel corner: v -> -v - 1
    t0 = {tuple(o): k for o, k in zip(o0.tolist(), c0.tolist())}
    assert all(t0[tuple(-np.array(o) - 1)] == k for o, k in t0.items())


# ---------------------------------------------------------------- Nyquist reading
def test_nyquist_reading_equals_half_spectrum_with_averaged_operator():
    """On even edges the real part of the inverse equals applying, on the Nyquist
    planes, the average of the operator over the sign of the Nyquist components."""
    n = (8, 6, 10)
    rng = np.random.default_rng(6)
    eps = rng.normal(size=(6,) + n)
    ref = O.solve_stress(eps, C_CUBIC, H, O.MEAN_STRESS_ZERO)
    eh = np.fft.rfftn(eps, axes=(3, 2, 1))        # half spectrum along x (axis 1)
    eh = np.fft.rfftn(eps.transpose(0, 3, 2, 1), axes=(1, 2, 3))  # (6, nz, ny, nx//2+1)
    nz, ny, nxh = eh.shape[1:]
    out = np.zeros_like(eh)
    for kz in range(nz):
        for ky in range(ny):
            for kx in range(nxh):
                fr = np.array([kx if kx < n[0] // 2 else -n[0] // 2,
                               ky if ky < n[1] // 2 else ky - n[1],
                               kz if kz < n[2] // 2 else kz - n[2]], dtype=float)
                nyq = np.array([kx == n[0] // 2, ky == n[1] // 2, kz == n[2] // 2])
                xi = 2 * np.pi * fr / (np.array(n) * H)
                e3 = O.to_tensor(eh[:, kz, ky, kx])[:, :, None]
                zero = np.array([not xi.any()])
                s = O.green_sigma_hat(C_CUBIC, xi[None], e3, O.MEAN_STRESS_ZERO, zero)
                if nyq.any():
                    xi2 = np.where(nyq, -xi, xi)
                    s = 0.5 * (s + O.green_sigma_hat(C_CUBIC, xi2[None], e3, O.MEAN_STRESS_ZERO, zero))
                out[:, kz, ky, kx] = O.to_voigt6(s[:, :, 0])
    sig = np.fft.irfftn(out, s=(n[2], n[1], n[0]), axes=(1, 2, 3)).transpose(0, 3, 2, 1)
    assert np.abs(sig - ref).max() < 1e-12 * np.abs(ref).max()


# ---------------------------------------------------------------- kinetics
def test_philox_known_answers():
    with open(os.path.join(GOLD, 'philox4x32_10_kat.txt')) as f:
        for line in f:
            if line.startswith('#') or not line.strip():
                continue
            w = [int(t, 16) for t in line.split()]
            assert O.philox4x32_10(w[0:4], w[4:6]) == w[6:10]


def test_u53_range():
    assert O.u53(0, 0) == 2.0 ** -53
    assert O.u53(0xFFFFFFFF, 0xFFFFFFFF) == 1.0


def test_p12_unbiased_walk_msd_and_residence_time():
    """No interaction: every jump of a 3D walker is (+-1,+-1,+-1) half-lattice units, so
    E|X_K|^2 = 3K (Var = 6K^2 per walker), and the mean residence time is 1/R_tot."""
    n = (1000, 1000, 1000)
    T = 300.0
    E = np.zeros(1)
    Ec = np.zeros((1, 8))
    W, K = 200, 100
    msd, dts = [], []
    for w in range(W):
        d = make_defects([O.SIA_CLUSTER], np.array([[1, 1, 1]]), [0], [0.0], [1], [0.34], [O.THREE_D])
        disp = np.zeros(3, dtype=np.int64)
        for step in range(K):
            i, j, dt, R = O.residence_step(d, E, Ec, T, 1000 + w, step, n)
            dts.append(dt)
            disp += O.JUMPS[j]
        msd.append(float(disp @ disp))
    nu = O.nominal_frequency(0.34, T)
    assert abs(R - nu) < 1e-9 * nu                    # z = 8 jumps at nu/8 each
    assert abs(np.mean(dts) - 1.0 / R) < 5.0 / R / np.sqrt(W * K)
    assert abs(np.mean(msd) - 3 * K) < 5 * np.sqrt(6.0) * K / np.sqrt(W)


def test_p12_p14_paper_time_step():
    g = json.load(open(os.path.join(GOLD, 'paper_table1.json')))
    d = make_defects([O.LOOP_111], np.array([[0, 0, 0]]), [0], [1.0], [0], [g['dl_Em_eV']], [O.ONE_D])
    dt = O.fixed_dt(d, g['dl_T_K'])
    assert abs(dt * 1e12 - g['dl_time_step_ps']) < 0.01


def test_p13_detailed_balance_on_ring():
    """Stationary occupancy of a ring with a frozen potential is Boltzmann."""
    K = 12
    T = 400.0
    rng = np.random.default_rng(7)
    Ek = rng.normal(scale=0.05, size=K)
    Q = np.zeros((K, K))
    for k in range(K):
        for step, jj in ((1, 7), (-1, 0)):          # jumps +lambda / -lambda on the ring
            Ec = np.zeros(8)
            Ec[jj] = Ek[(k + step) % K]
            allowed = np.zeros(8, bool)
            allowed[[0, 7]] = True
            Ec[7 - jj] = Ek[(k - step) % K]
            r = O.jump_rates(0.2, Ek[k], Ec, allowed, T)
            Q[k, (k + step) % K] += r[jj]
    np.fill_diagonal(Q, -Q.sum(axis=1))
    A = np.vstack([Q.T, np.ones(K)])
    b = np.zeros(K + 1)
    b[-1] = 1.0
    pi = np.linalg.lstsq(A, b, rcond=None)[0]
    boltz = np.exp(-Ek / (O.KB * T))
    boltz /= boltz.sum()
    assert np.abs(pi - boltz).max() < 1e-12


def test_selection_rule_boundaries():
    rates = np.array([1.0, 2.0, 0.0, 1.0])
    assert O.select_on_line(rates, 0.25)[0] == 0       # R_0/R = 0.25 -> inclusive on the right
    assert O.select_on_line(rates, 0.2500001)[0] == 1
    assert O.select_on_line(rates, 0.75)[0] == 1
    assert O.select_on_line(rates, 0.7500001)[0] == 3  # zero-rate entry never selected
    assert O.select_on_line(rates, 1.0)[0] == 3


def test_fixed_dt_step_moves_only_mobile():
    d = make_defects([O.LOOP_111, O.LOOP_100], np.array([[0, 0, 0], [10, 10, 10]]), [0, 0],
                     [1.0, 1.0], [0, 0], [0.1, 1.0], [O.ONE_D, O.IMMOBILE])
    dt = O.fixed_dt(d, 300.0)
    moved = 0
    for step in range(200):
        mv = O.fixed_dt_step(d, np.zeros(2), np.zeros((2, 8)), 300.0, 99, step, (64, 64, 64), dt)
        moved += len(mv)
        assert all(i == 0 for i, _ in mv)
    # the fastest defect jumps with probability 1 - e^-1 per step
    assert abs(moved / 200 - (1 - np.exp(-1))) < 4 * np.sqrt(0.25 / 200)
    assert np.array_equal(d['pos'][1], [10, 10, 10])


# ---------------------------------------------------------------- P14: Table 1
def test_p14_table1_conversions():
    g = json.load(open(os.path.join(GOLD, 'paper_table1.json')))
    E, nu = O.zener_isotropic_moduli(g['C11_GPa'], g['C12_GPa'])
    assert abs(E - g['E_iso_GPa']) < 0.01 and abs(nu - g['nu_iso']) < 1e-3
    a0 = g['a0_A'] / 10.0                      # nm
    omega = a0 ** 3 / 2.0
    assert abs(omega * 1000 - g['V_at_A3']) < 0.01
    b = math.sqrt(3.0) / 2.0 * a0
    r = math.sqrt(800 * omega / b / math.pi) * 10.0
    assert abs(r - g['loop_800_SIA_radius_A']) < g['loop_radius_rel_tol'] * g['loop_800_SIA_radius_A']
    P = g['P_SIA_eV']
    B = (g['C11_GPa'] + 2 * g['C12_GPa']) / 3.0
    dv = (P['P11'] + P['P22'] + P['P33']) / O.KAPPA / (3 * B)      # nm^3
    assert abs(dv / omega - g['relaxation_volume_over_Vat']) < 2e-3
    # the oracle's copy of the tensor, in (xx, yy, zz, yz, xz, xy) order
    assert np.array_equal(O.SIA_110_DIPOLE_EV, [P['P11'], P['P22'], P['P33'], P['P23'], P['P13'], P['P12']])


# ---------------------------------------------------------------- dipole approximation
# Sec. 2.1, Eqs. interaction_energy4 and dipole_def2: E_dip_i(Y) = -(int eps*_i) : sigma^(-i)(Y)
def test_dipole_self_table_fourier_equals_real_space():
    """The self part D(c, k) by Fourier sums equals the single-defect solve sampled at the
    centres (two independent routes)."""
    n = (16, 16, 16)
    for d in _defects_small():
        D = O.dipole_self_table(d, n, H, C_CUBIC)
        Df = O.dipole_self_table_fourier(d, n, H, C_CUBIC)
        assert np.abs(D - Df).max() <= 1e-10 * np.abs(D).max()


def test_dipole_table_route_equals_bruteforce():
    """kappa (int eps*) : sigma(Y) minus the translation-invariant self part equals the
    energy against sigma - sigma_i (the route the CUDA path takes)."""
    n = (16, 16, 16)
    d = _defects_small()
    E, Ec = O.dipole_energies(d, n, H, C_CUBIC)
    sig = O.solve_stress(O.eigenstrain_field(d, n, H), C_CUBIC, H)
    for i in range(len(d)):
        D = O.dipole_self_table(d[i], n, H, C_CUBIC)
        c = O.pos_class(d[i]['pos'])
        ie = O.integrated_eigenstrain6(d[i], H)
        e0 = -O.KAPPA * (O.ddot6(ie, O.sample_center(sig, d[i]['pos'])) - D[c, 0])
        assert abs(e0 - E[i]) <= 1e-10 * max(1.0, O.KAPPA * np.abs(D).max())
        for j, Y in enumerate(O.candidate_positions(d[i]['pos'])):
            ej = -O.KAPPA * (O.ddot6(ie, O.sample_center(sig, Y)) - D[c, 1 + j])
            assert abs(ej - Ec[i, j]) <= 1e-10 * max(1.0, O.KAPPA * np.abs(D).max())


def test_dipole_equals_exact_when_the_stencil_is_the_centre_sample():
    """A cluster whose stencil at a class-0 site is the 8 voxels around its centre with
    equal weights: the exact energy (Eq. interaction_energy3) averages sigma^(-i) over
    exactly the voxels whose mean is the dipole sample, so the two agree."""
    n = (16, 16, 16)
    d = _defects_small()
    offs, cnt, _ = O.stencil(d[2], 0, H)
    assert len(cnt) == 8 and np.all(cnt == cnt[0])
    assert sorted(map(tuple, offs)) == sorted(map(tuple, O.center_voxels(np.zeros(3, np.int64))))
    E, _ = O.dipole_energies(d, n, H, C_CUBIC)
    Ex, _ = O.energies_bruteforce(d, n, H, C_CUBIC)
    assert abs(E[2] - Ex[2]) <= 1e-12 * abs(Ex[2])
    assert abs(E[0] - Ex[0]) > 1e-3 * abs(Ex[0])        # a loop is not a point defect


def test_dipole_approaches_exact_with_separation():
    """Two small loops along a ray: the relative gap between the dipole and the exact
    interaction energies falls as the separation grows (Sec. 6: the dipole form holds
    for sufficiently far defects)."""
    N = 48
    n = (N, N, N)
    gaps = []
    for step in (3, 5, 8):
        p1 = np.array([N, N, N])
        p2 = p1 + step * np.array([2, 2, 0])
        d = [dict(type=O.LOOP_111, pos=p1, axis=0, radius_nm=0.45, size=0, Em_eV=0.1, mobility=O.ONE_D),
             dict(type=O.LOOP_111, pos=p2, axis=1, radius_nm=0.45, size=0, Em_eV=0.1, mobility=O.ONE_D)]
        E, _ = O.dipole_energies(d, n, H, C_CUBIC)
        Ex, _ = O.energies_bruteforce(d, n, H, C_CUBIC)
        gaps.append(abs(E[1] - Ex[1]) / abs(Ex[1]))
    assert gaps[0] > gaps[1] > gaps[2], gaps
    assert gaps[2] < 0.08, gaps


def test_dipole_limit_isotropic_kelvin():
    """Isotropic medium: energy changes of a small loop's dipole energy along a ray follow
    the Kelvin dipole-dipole expression P1_ij P2_kl d_j d_l G_ik (cf. P8)."""
    mu, nu = 82.0, 0.29
    C = O.stiffness_cubic(*O.isotropic_cubic_constants(mu, nu))
    N = 96
    n = (N, N, N)
    c0 = np.array([N, N, N])
    loop = dict(type=O.LOOP_111, pos=c0, axis=0, radius_nm=0.35, size=0, Em_eV=0.1, mobility=O.ONE_D)
    eps = O.eigenstrain_field([loop], n, H)
    s0 = O.solve_stress(eps, C, H, O.MEAN_STRAIN_ZERO)
    P = np.einsum('ijkl,kl->ij', C, O.to_tensor(eps.reshape(6, -1).sum(axis=1) * H ** 3))
    rows = []
    for step in (8, 10, 12, 14):
        p2 = c0 + step * np.array([2, 1, -1])
        rows.append((O.dipole_energy_at(loop, p2, s0, H),
                     O.dipole_dipole_energy(P, P, (p2 - c0) * H / 2.0, mu, nu) * O.KAPPA))
    errs = [abs((rows[k + 1][0] - rows[k][0]) / (rows[k + 1][1] - rows[k][1]) - 1.0) for k in range(len(rows) - 1)]
    assert all(errs[k + 1] < errs[k] for k in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-2, errs


def test_blin_far_field_is_the_kelvin_dipole_dipole_energy():
    """Blin's double line integral for two loops (prismatic/prismatic with different
    Burgers vectors, prismatic/shear, shear/shear) approaches the Kelvin dipole-dipole
    energy of their dipole tensors P = C : sym(b (x) A) as the separation grows, the gap
    falling like (R/d)^2 (a factor of about 4 per doubling); all three of its terms
    contribute across these pairs."""
    mu, nu, R = 82.0, 0.29, 0.7
    C = O.stiffness_cubic(*O.isotropic_cubic_constants(mu, nu))
    pairs = [([1, 1, 1], [1, 1, 1], [-1, 1, 1], [-1, 1, 1]), ([1, 1, 1], [1, 1, 1], [1, 1, 1], [1, -1, 0]),
             ([1, 0, 0], [0, 1, 1], [0, 1, 0], [1, 0, 1])]
    for b1, n1, b2, n2 in pairs:
        b1, b2 = 0.25 * np.array(b1) / np.linalg.norm(b1), 0.25 * np.array(b2) / np.linalg.norm(b2)
        n1, n2 = np.array(n1) / np.linalg.norm(n1), np.array(n2) / np.linalg.norm(n2)
        P1 = O.loop_dipole_tensor(C, b1, PI_ * R * R * n1)
        P2 = O.loop_dipole_tensor(C, b2, PI_ * R * R * n2)
        gaps = []
        for dist in (10.0, 20.0, 40.0):
            d = dist * np.array([2.0, 1.0, -1.0]) / np.sqrt(6.0)
            w = O.blin_interaction_energy(O.circle_points(np.zeros(3), n1, R, 400), b1,
                                          O.circle_points(d, n2, R, 400), b2, mu, nu)
            gaps.append(abs(w / O.dipole_dipole_energy(P1, P2, d, mu, nu) - 1.0))
        assert gaps[2] < 0.02 and gaps[1] / gaps[2] > 3.0 and gaps[0] / gaps[1] > 3.0, gaps


def test_p9_near_field_converges_to_blin():
    """Near field (Sec. 2, Eq. interaction_energy3 by the periodic solve) against Blin's
    infinite-body energy for two prismatic 1/2<111> loops (R = 0.7 nm, isotropic) whose
    centres are 2.28 and 3.43 nm apart along [100], where the dipole form is off by 85%:
    in a fixed 13.7 nm box refined from h = 0.29 to 0.14 nm (b = (a0/2)[111] with
    a0 = h), the change of energy between the two separations (which cancels the
    box's uniform image term) approaches Blin's monotonically, roughly linearly in h
    (the slab's thickness), and extrapolates to it within 2%."""
    mu, nu, R = 82.0, 0.29, 0.7
    C = O.stiffness_cubic(*O.isotropic_cubic_constants(mu, nu))
    n111 = np.ones(3) / np.sqrt(3.0)
    Lbox = 48 * H
    hs, errs = [], []
    for N, k1, k2 in ((48, 8, 12), (72, 12, 18), (96, 16, 24)):
        h = Lbox / N
        n = (N, N, N)
        c = np.array([N, N, N])
        b = (np.sqrt(3.0) / 2.0) * h * n111
        loops = [dict(type=O.LOOP_111, pos=c + np.array([2 * k, 0, 0]), axis=0, radius_nm=R, size=0, Em_eV=0.1,
                      mobility=O.ONE_D) for k in (0, k1, k2)]
        E, W = [], []
        for l2 in loops[1:]:
            s2 = O.solve_stress(O.eigenstrain_field([l2], n, h), C, h)
            E.append(O.energy_of_stencil(loops[0], loops[0]['pos'], s2, h))
            W.append(O.KAPPA * O.blin_interaction_energy(O.circle_points(c * h / 2, n111, R, 600), b,
                                                         O.circle_points(l2['pos'] * h / 2, n111, R, 600), b, mu, nu))
        hs.append(h)
        errs.append((E[0] - E[1]) / (W[0] - W[1]) - 1.0)
    assert abs(errs[0]) > abs(errs[1]) > abs(errs[2]), errs
    slope = (errs[1] - errs[2]) / (hs[1] - hs[2])
    assert abs(errs[2] - slope * hs[2]) < 0.02, errs


def test_point_dipole_energy_closed_forms_and_defect_dipole():
    """E = -P : C^-1 : sigma for a given dipole tensor (Table 1's <110> dumbbell):
    under a uniform hydrostatic stress p it is -tr(P) p / (3K), K = (C11 + 2 C12)/3;
    under a uniform shear sigma_yz = tau it is -P_yz tau / C44; and with the defect's own
    dipole tensor P = kappa C : int eps* it equals the defect's dipole energy
    -kappa (int eps*) : sigma at every site."""
    C11, C12, C44 = 289.34, 152.34, 107.43     # Table 1
    C = O.stiffness_cubic(C11, C12, C44)
    P = O.SIA_110_DIPOLE_EV
    n = (8, 8, 8)
    p, tau = 0.7, -0.3
    hyd = np.zeros((6,) + n)
    hyd[:3] = p
    K = (C11 + 2.0 * C12) / 3.0
    for pos in ([2, 4, 6], [3, 5, 7]):
        assert abs(O.point_dipole_energy(P, np.array(pos), hyd, C) + P[:3].sum() * p / (3.0 * K)) < 1e-12
    sh = np.zeros((6,) + n)
    sh[3] = tau
    assert abs(O.point_dipole_energy(P, np.array([2, 4, 6]), sh, C) + P[3] * tau / C44) < 1e-12
    rng = np.random.default_rng(5)
    sig = rng.normal(size=(6,) + n)
    loop = dict(type=O.LOOP_111, pos=np.array([6, 8, 4]), axis=2, radius_nm=0.4, size=0, Em_eV=0.1, mobility=O.ONE_D)
    Pd = O.KAPPA * (O.stiffness_matrix(C) @ (O.integrated_eigenstrain6(loop, H) * np.array([1, 1, 1, 2, 2, 2])))
    for pos in ([6, 8, 4], [7, 9, 5], [1, 3, 15]):
        a = O.point_dipole_energy(Pd, np.array(pos), sig, C)
        b = O.dipole_energy_at(loop, np.array(pos), sig, H)
        assert abs(a - b) <= 1e-12 * abs(b)


# ---------------------------------------------------------------- dislocation lines (FDM)
# Sec. 3.2, Eqs. Nye2, curlUe, eq_EIG_fourier, plastic_0
def _edge_dislocation_stress(N, mu, nu, b=0.25):
    """Stress of a straight edge dislocation (line along z through a voxel corner at the
    box centre, b along x) by the FDM route, and the Volterra isotropic solution at the
    voxel centres (Hirth & Lothe, Eq. 3-43)."""
    C = O.stiffness_cubic(*O.isotropic_cubic_constants(mu, nu))
    n = (N, N, N)
    x0 = np.array([N / 2 * H, N / 2 * H, 0.0])
    bv = np.array([b, 0.0, 0.0])
    alpha = O.nye_tensor(np.array([x0, x0 + np.array([0.0, 0.0, N * H])]), bv, n, H, closed=False)
    s = O.solve_stress(O.dislocation_eigenstrain6(alpha, H), C, H).reshape(6, -1)
    xc = (np.indices(n).reshape(3, -1).T + 0.5) * H
    x, y = xc[:, 0] - x0[0], xc[:, 1] - x0[1]
    r4 = (x * x + y * y) ** 2
    D = mu * b / (2.0 * PI_ * (1.0 - nu))
    v = np.zeros_like(s)
    v[0] = -D * y * (3 * x * x + y * y) / r4
    v[1] = D * y * (x * x - y * y) / r4
    v[5] = D * x * (x * x - y * y) / r4
    v[2] = nu * (v[0] + v[1])
    return s, v, np.hypot(x, y)


PI_ = math.pi


def test_fdm_edge_dislocation_matches_volterra():
    """Isotropic medium: near the core (far from the periodic images) the FDM stress of a
    straight edge dislocation is Volterra's; the gap further out falls as the box grows
    (the images and the uniform compensating density of a net Burgers vector)."""
    mu, nu = 82.0, 0.29
    s64, v64, r64 = _edge_dislocation_stress(64, mu, nu)
    m = (r64 >= 0.8) & (r64 < 2.5)
    assert np.linalg.norm(s64[:, m] - v64[:, m]) <= 0.06 * np.linalg.norm(v64[:, m])
    s96, v96, r96 = _edge_dislocation_stress(96, mu, nu)
    far = [np.linalg.norm(s[:, (r >= 2.5) & (r < 4.0)] - v[:, (r >= 2.5) & (r < 4.0)])
           / np.linalg.norm(v[:, (r >= 2.5) & (r < 4.0)]) for s, v, r in ((s64, v64, r64), (s96, v96, r96))]
    assert far[1] < 0.6 * far[0], far


def test_fdm_screw_dislocation_along_a_cube_axis_matches_the_antiplane_solution():
    """A screw dislocation along [001] of a cubic crystal is an antiplane problem with
    modulus C44 exactly (no coupling through C11 or C12): sigma_xz = -C44 b y / (2 pi r^2),
    sigma_yz = C44 b x / (2 pi r^2), every other component zero (Hirth & Lothe Eq. 3-3 with
    mu = C44).  The FDM route with the anisotropic Green operator gives it within a few
    per cent next to the core, the in-plane stresses vanish to rounding, and the gap
    further out falls as the box grows."""
    C11, C12, C44, b = 243.0, 145.0, 116.0, 0.25
    C = O.stiffness_cubic(C11, C12, C44)
    gaps = []
    for N in (64, 96):
        n = (N, N, N)
        x0 = np.array([N / 2 * H, N / 2 * H, 0.0])
        alpha = O.nye_tensor(np.array([x0, x0 + np.array([0.0, 0.0, N * H])]), np.array([0.0, 0.0, b]), n, H,
                             closed=False)
        s = O.solve_stress(O.dislocation_eigenstrain6(alpha, H), C, H).reshape(6, -1)
        xc = (np.indices(n).reshape(3, -1).T + 0.5) * H
        x, y = xc[:, 0] - x0[0], xc[:, 1] - x0[1]
        r2 = x * x + y * y
        v = np.zeros_like(s)
        v[4] = -C44 * b * y / (2.0 * PI_ * r2)
        v[3] = C44 * b * x / (2.0 * PI_ * r2)
        r = np.sqrt(r2)
        near, far = (r >= 0.8) & (r < 2.5), (r >= 2.5) & (r < 4.0)
        assert np.abs(s[[0, 1, 2, 5]]).max() < 1e-12 * np.abs(s).max()
        gaps.append([np.linalg.norm(s[:, m] - v[:, m]) / np.linalg.norm(v[:, m]) for m in (near, far)])
    assert gaps[0][0] < 0.04 and gaps[1][0] < gaps[0][0], gaps
    assert gaps[1][1] < 0.6 * gaps[0][1], gaps


def test_fdm_loop_nye_tensor_moments_and_mean():
    """A closed loop's Nye tensor integrates to zero, its first moment is b (x) (oriented
    area) (the loop's dipole), and the compatible part of Eq. plastic_0 gives the mean
    eigenstrain sym(b (x) A)/V, the slab loop's integrated eigenstrain over the box."""
    N = 32
    n = (N, N, N)
    pos = np.array([N, N, N])
    R = 1.0
    loop = dict(type=O.LOOP_111, pos=pos, axis=0, radius_nm=R, size=0, Em_eV=0.1, mobility=O.ONE_D)
    g = O.defect_geometry(loop, H)
    X = pos * H / 2.0
    alpha = O.nye_tensor(O.circle_points(X, g['n'], R, 1024)[::-1], g['b'], n, H)
    assert np.abs(alpha.reshape(9, -1).sum(axis=1)).max() * H ** 3 < 1e-12
    d = (np.indices(n).reshape(3, -1).T + 0.5) * H - X
    M = np.einsum('ilv,vm->ilm', alpha.reshape(3, 3, -1), d) * H ** 3          # int alpha_il x_m
    A = PI_ * R * R * g['n']
    # clockwise line seen from A's tip (curl U^p = -alpha with U^p = b (x) n on the loop's
    # surface): int alpha_il x_m = b_i eps_lmp A'_p, A' the inscribed 1024-gon's area vector
    Ap = A * (1024 / (2.0 * PI_)) * math.sin(2.0 * PI_ / 1024)
    expect = np.einsum('i,lmp,p->ilm', g['b'], O.LEVI_CIVITA, Ap)
    assert np.abs(M - expect).max() <= 1e-9 * np.abs(expect).max()
    U0 = 0.5 * (np.outer(g['b'], A) + np.outer(A, g['b'])) / (np.prod(n) * H ** 3)
    eps = O.dislocation_eigenstrain6(alpha, H, U0)
    slab = O.eigenstrain_field([loop], n, H)
    assert np.allclose(eps.reshape(6, -1).sum(axis=1), slab.reshape(6, -1).sum(axis=1), rtol=1e-10, atol=1e-12)


def test_fdm_nye_tensor_moments_of_arbitrary_closed_lines():
    """For any closed polyline (here non-planar random ones, away from the box edges) the
    spread Nye tensor integrates to zero and its first moment is b_i oint x_m dx_l =
    b_i eps_mlp A_p with A = 1/2 oint x x dx: trilinear spreading keeps first moments and
    the midpoint rule is exact on straight segments."""
    rng = np.random.default_rng(11)
    n = (24, 24, 24)
    centre = np.full(3, 12 * H)
    for trial in range(3):
        pts = centre + rng.normal(scale=0.6, size=(int(rng.integers(5, 12)), 3))
        b = rng.normal(size=3) * 0.2
        alpha = O.nye_tensor(pts, b, n, H, closed=True)
        assert np.abs(alpha.reshape(9, -1).sum(axis=1)).max() * H ** 3 < 1e-12
        x = (np.indices(n).reshape(3, -1).T + 0.5) * H
        M = np.einsum('ilv,vm->ilm', alpha.reshape(3, 3, -1), x) * H ** 3
        A = 0.5 * np.sum(np.cross(pts, np.roll(pts, -1, axis=0)), axis=0)
        expect = np.einsum('i,mlp,p->ilm', b, O.LEVI_CIVITA, A)
        assert np.abs(M - expect).max() <= 1e-10 * max(1.0, np.abs(expect).max()), trial


def test_fdm_loop_approaches_slab_loop_with_resolution():
    """The same prismatic loop as a line (Nye tensor, this route) and as the one-voxel
    slab of Eq. eig_shearloop: a loop's stress depends on its line only, so away from the
    core the two fields approach each other as the voxel shrinks in a fixed box."""
    Lbox, R = 32 * H, 1.2
    C = C_CUBIC
    gaps = []
    for N in (24, 32, 48):
        h = Lbox / N
        n = (N, N, N)
        pos = np.array([N, N, N])
        loop = dict(type=O.LOOP_111, pos=pos, axis=0, radius_nm=R, size=0, Em_eV=0.1, mobility=O.ONE_D)
        g = O.defect_geometry(loop, h)
        X = pos * h / 2.0
        s_slab = O.solve_stress(O.eigenstrain_field([loop], n, h), C, h).reshape(6, -1)
        alpha = O.nye_tensor(O.circle_points(X, g['n'], R, 1024)[::-1], g['b'], n, h)
        s_fdm = O.solve_stress(O.dislocation_eigenstrain6(alpha, h), C, h).reshape(6, -1)
        d = (np.indices(n).reshape(3, -1).T + 0.5) * h - X
        r = np.linalg.norm(d - np.round(d / Lbox) * Lbox, axis=1)
        m = (r >= 2.0) & (r < 3.5)
        gaps.append(np.linalg.norm(s_slab[:, m] - s_fdm[:, m]) / np.linalg.norm(s_slab[:, m]))
    assert gaps[0] > gaps[1] > gaps[2], gaps
    assert gaps[2] < 0.35, gaps


# ---------------------------------------------------------------- shift theorem (Sec. 3.3, Eq. shift)
def _paper_form_direct(d, i, n, C):
    """kappa int sigma_ext : eps^{i,e} with defect i rasterised at its position."""
    s_ext = O.solve_stress(O.eigenstrain_field(d, n, H, exclude={i}), C, H)
    s_i = O.solve_stress(O.eigenstrain_field(d, n, H, only={i}), C, H)
    S = np.linalg.inv(O.stiffness_matrix(C))
    e = np.einsum('ab,b...->a...', S, s_i)
    e[3:] *= 0.5
    return s_ext, O.KAPPA * H ** 3 * np.sum(O.ddot6(s_ext, e))


@pytest.mark.parametrize('n', [(15, 15, 15), (16, 16, 16)])
def test_shift_theorem_whole_voxel_shift_equals_rasterised(n):
    """A reference field moved by a whole-voxel vector (Eq. shift) is the defect rasterised
    there: same paper-form energy; on odd edges also the eigenstrain-form energy."""
    d = _defects_small()
    E, _ = O.energies_bruteforce(d, n, H, C_CUBIC)
    for i in (0, 2):                                  # class-0 sites
        s_ext, e_dir = _paper_form_direct(d, i, n, C_CUBIC)
        ref = O.elastic_strain_spectrum(d[i], n, H, C_CUBIC)
        e_sh = O.energy_shift_theorem(ref, np.asarray(d[i]['pos']) * H / 2.0, s_ext, H)
        assert abs(e_sh - e_dir) <= 1e-10 * max(1.0, abs(e_dir))
        if n[0] % 2:
            assert abs(e_sh - E[i]) <= 1e-10 * max(1.0, abs(E[i]))


def test_shift_theorem_routes_agree_and_uniform_field_is_position_independent():
    """At continuous positions the Parseval sum equals the explicit inverse transform of
    the moved field, and in a uniform external stress the energy does not depend on X."""
    n = (16, 16, 16)
    d = _defects_small()
    ref = O.elastic_strain_spectrum(d[0], n, H, C_CUBIC)
    s_ext = O.solve_stress(O.eigenstrain_field(d, n, H, exclude={0}), C_CUBIC, H)
    rng = np.random.default_rng(5)
    for X in rng.uniform(0.0, 16 * H, size=(3, 3)):
        e1 = O.energy_shift_theorem(ref, X, s_ext, H)
        e2 = O.KAPPA * H ** 3 * np.sum(O.ddot6(s_ext, O.shifted_field(ref[1], X - ref[0], H)))
        assert abs(e1 - e2) <= 1e-10 * max(1.0, abs(e1))
    uniform = np.broadcast_to(np.array([1.0, -0.5, 0.3, 0.2, -0.1, 0.4])[:, None, None, None], (6,) + n).copy()
    vals = [O.energy_shift_theorem(ref, X, uniform, H) for X in rng.uniform(0.0, 16 * H, size=(4, 3))]
    assert max(vals) - min(vals) <= 1e-12 * max(1.0, abs(vals[0]))
