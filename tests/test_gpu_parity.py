"""GPU (CUDA library through the C ABI) versus the CPU FP64 oracle.

Bars: stencils bit exact; stress relative L2 <= 1e-5 (FP32 fields) or 1e-10 (FP64
fields); energies within 1e-4 eV (FP32) or 1e-8 eV (FP64); kinetic decisions equal
given the same energies and Philox counters.
"""
import time

import numpy as np
import pytest

import __graft_entry__
import oracle as O
from paper_2403_09158_gb300 import okmc as ok
from paper_2403_09158_gb300.workload import (DEFECT_DTYPE, FE_CUBIC, FE_ISO, config_large, config_medium, config_small,
                                             make_defects, scaled_population)

pytestmark = pytest.mark.gpu

STRESS_TOL = {ok.FP32_FIELDS: 1e-5, ok.FP64_FIELDS: 1e-10}
ENERGY_TOL = {ok.FP32_FIELDS: 1e-4, ok.FP64_FIELDS: 1e-8}


@pytest.fixture(scope='module', autouse=True)
def _lib():
    __graft_entry__.build()
    ok.load()


def zyx(a):
    """oracle (6, nx, ny, nz) -> library layout (6, nz, ny, nx)"""
    return np.transpose(a, (0, 3, 2, 1))


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def make_grid(w, precision=ok.FP32_FIELDS, k0=ok.MEAN_STRESS_ZERO, C=None, seed=11):
    C = C or w.C
    g = ok.Grid(w.n, w.voxel_nm, *C, k0_mode=k0, precision=precision, seed=seed)
    g.set_defects(w.defects)
    return g


# ------------------------------------------------------------------ stencils
def test_stencils_bit_exact():
    w = config_small()
    extra = make_defects([0, 0, 1, 1, 2, 2], np.array([[2, 2, 2], [5, 7, 9], [4, 6, 8], [3, 3, 3], [0, 0, 0], [1, 1, 1]]),
                         [1, 3, 0, 2, 0, 0], [1.37, 0.5, 0.9, 2.2, 0, 0], [0, 0, 0, 0, 1, 37],
                         [0.1, 0.1, 1, 1, 0.3, 0.3], [1, 1, 0, 0, 2, 1])
    defs = np.concatenate([w.defects, extra])
    g = ok.Grid((48, 48, 48), w.voxel_nm, *w.C)
    g.set_defects(defs)
    for i, d in enumerate(defs):
        for c in (0, 1):
            offs, cnt, alpha = g.stencil(i, c)
            o2, c2, a2 = O.stencil(d, c, w.voxel_nm)
            assert np.array_equal(offs, o2), (i, c)
            assert np.array_equal(cnt, c2), (i, c)
            assert abs(alpha - a2) <= 1e-15 * a2
    g.close()


# ------------------------------------------------------------------ eigenstrain and stress
@pytest.mark.parametrize('precision', [ok.FP32_FIELDS, ok.FP64_FIELDS])
def test_eigenstrain_field(precision):
    w = config_small()
    g = make_grid(w, precision)
    eps = g.eigenstrain()
    ref = zyx(O.eigenstrain_field(w.defects, w.n, w.voxel_nm))
    tol = 2e-7 if precision == ok.FP32_FIELDS else 1e-11
    assert np.abs(eps - ref).max() < tol
    g.close()


CASES = [
    ((32, 32, 32), ok.FP32_FIELDS, ok.MEAN_STRESS_ZERO, 'cubic', 12),
    ((32, 32, 32), ok.FP64_FIELDS, ok.MEAN_STRESS_ZERO, 'cubic', 12),
    ((32, 32, 32), ok.FP32_FIELDS, ok.MEAN_STRAIN_ZERO, 'iso', 12),
    ((16, 16, 16), ok.FP32_FIELDS, ok.MEAN_STRESS_ZERO, 'cubic', 3),
    ((48, 32, 80), ok.FP32_FIELDS, ok.MEAN_STRESS_ZERO, 'cubic', 20),
    ((80, 48, 32), ok.FP64_FIELDS, ok.MEAN_STRAIN_ZERO, 'cubic', 20),
    ((96, 64, 160), ok.FP32_FIELDS, ok.MEAN_STRESS_ZERO, 'cubic', 30),
    ((64, 64, 64), ok.FP64_FIELDS, ok.MEAN_STRESS_ZERO, 'iso', 25),
    # register-FFT passes with mixed-radix lines (2^a 3^b 5^c)
    ((48, 48, 48), ok.FP32_FIELDS, ok.MEAN_STRESS_ZERO, 'cubic', 15),
    ((96, 96, 96), ok.FP32_FIELDS, ok.MEAN_STRAIN_ZERO, 'iso', 30),
    ((160, 160, 32), ok.FP32_FIELDS, ok.MEAN_STRESS_ZERO, 'cubic', 30),
    ((192, 192, 48), ok.FP32_FIELDS, ok.MEAN_STRESS_ZERO, 'cubic', 30),
    ((320, 320, 32), ok.FP32_FIELDS, ok.MEAN_STRAIN_ZERO, 'cubic', 30),
    ((32, 32, 320), ok.FP32_FIELDS, ok.MEAN_STRESS_ZERO, 'cubic', 20),
    ((64, 64, 192), ok.FP32_FIELDS, ok.MEAN_STRESS_ZERO, 'cubic', 20),
]
FAST_EDGES = {32, 48, 64, 96, 128, 160, 192, 256, 320}


@pytest.mark.parametrize('n,precision,k0,mat,nd', CASES)
def test_stress_parity(n, precision, k0, mat, nd):
    w = scaled_population(n, nd, seed=sum(n) + nd, r111=(0.4, 1.0), r100=(0.4, 1.0))
    C = FE_CUBIC if mat == 'cubic' else O.isotropic_cubic_constants(*FE_ISO)
    g = make_grid(w, precision, k0, C)
    fast = precision == ok.FP32_FIELDS and n[0] == n[1] and n[0] in FAST_EDGES and n[2] in FAST_EDGES
    assert (g.launch_shape()[0] == -1) == fast
    sig = g.solve_stress()
    ref = zyx(O.solve_stress(O.eigenstrain_field(w.defects, w.n, w.voxel_nm), O.stiffness_cubic(*C),
                             w.voxel_nm, k0))
    assert rel_l2(sig, ref) <= STRESS_TOL[precision]
    g.close()


# ------------------------------------------------------------------ energies
@pytest.mark.parametrize('precision', [ok.FP32_FIELDS, ok.FP64_FIELDS])
def test_energies_bruteforce_small(precision):
    w = config_small()
    g = make_grid(w, precision)
    E = g.interaction_energies()
    Ec, valid = g.candidate_energies()
    Eo, Eco = O.energies_bruteforce(w.defects, w.n, w.voxel_nm, O.stiffness_cubic(*w.C))
    tol = ENERGY_TOL[precision]
    assert np.abs(E - Eo).max() <= tol, np.abs(E - Eo).max()
    assert np.abs(Ec - Eco).max() <= tol, np.abs(Ec - Eco).max()
    for i, d in enumerate(w.defects):
        assert np.array_equal(valid[i].astype(bool), O.allowed_jumps(d))
    g.close()


@pytest.mark.parametrize('precision', [ok.FP32_FIELDS, ok.FP64_FIELDS])
def test_candidate_energies_large_loop_and_small_defects(precision):
    """A loop too large for the dilated candidate lists (scan box side 63 voxels) takes
    the direct candidate loop; the small defects beside it take the lists.  Both match
    the brute-force oracle (N_d + 1 solves)."""
    from paper_2403_09158_gb300.workload import LOOP_111, ONE_D, SIA_CLUSTER, THREE_D
    defs = make_defects([LOOP_111, SIA_CLUSTER, SIA_CLUSTER, LOOP_111],
                        np.array([[64, 64, 64], [10, 10, 100], [101, 21, 31], [30, 100, 20]]), [0, 1, 2, 3],
                        [8.2, 0.0, 0.0, 0.8], [0, 3, 1, 0], [0.1, 0.3, 0.3, 0.1], [ONE_D, ONE_D, THREE_D, ONE_D])
    n = (64, 64, 64)
    g = ok.Grid(n, 0.2855, *FE_CUBIC, precision=precision)
    g.set_defects(defs)
    E = g.interaction_energies()
    Ec, _ = g.candidate_energies()
    W = g.self_terms()
    g.close()
    Eo, Eco = O.energies_bruteforce(defs, n, 0.2855, O.stiffness_cubic(*FE_CUBIC))
    # the flat bar, although this loop's own field is extreme (R = 8.2 nm in an 18 nm
    # box; self term ~1.5e3 eV)
    tol = np.full(len(defs), ENERGY_TOL[precision])
    assert np.all(np.abs(E - Eo) <= tol), (np.abs(E - Eo), tol)
    assert np.all(np.abs(Ec - Eco).max(axis=1) <= tol), (np.abs(Ec - Eco).max(axis=1), tol)


def test_self_terms_match_oracle():
    w = config_small()
    g = make_grid(w, ok.FP64_FIELDS)
    W = g.self_terms()
    C = O.stiffness_cubic(*w.C)
    for i in (0, 2, 5):
        Wo = O.self_term_table_fourier(w.defects[i], w.n, w.voxel_nm, C)
        assert np.abs(W[i] - Wo).max() <= 1e-9 * max(1.0, np.abs(Wo).max())
    g.close()
    # FP32 spectra: the table inherits the transform's ~1e-7 relative error; what the
    # energies need is that error well under the 1e-4 eV bar
    g = make_grid(w, ok.FP32_FIELDS)
    W = g.self_terms()
    for i in (0, 2, 5):
        Wo = O.self_term_table_fourier(w.defects[i], w.n, w.voxel_nm, C)
        assert np.abs(W[i] - Wo).max() <= 5e-7 * np.abs(Wo).max() + 1e-6
        assert np.abs(W[i] - Wo).max() <= 5e-5
    g.close()


# ------------------------------------------------------------------ dipole approximation
@pytest.mark.parametrize('precision', [ok.FP32_FIELDS, ok.FP64_FIELDS])
def test_dipole_energies_match_oracle(precision):
    """Dipole-approximation energies (Eq. interaction_energy4, P = C : int eps*) at the
    sites and after the jumps, and their self part, against the oracle's sigma - sigma_i
    route and its Fourier table."""
    w = config_small()
    g = make_grid(w, precision)
    Ex = g.interaction_energies()
    E, Ec = g.dipole_energies()
    D = g.dipole_self_terms()
    # the tables are built on first use with the field buffers as scratch; the field is
    # rebuilt from the positions, so the exact energies do not change
    assert np.array_equal(g.interaction_energies(), Ex)
    g.close()
    C = O.stiffness_cubic(*w.C)
    Eo, Eco = O.dipole_energies(w.defects, w.n, w.voxel_nm, C)
    Do = np.array([O.dipole_self_table_fourier(d, w.n, w.voxel_nm, C) for d in w.defects])
    if precision == ok.FP64_FIELDS:
        assert np.abs(D - Do).max() <= 1e-9 * max(1.0, np.abs(Do).max())
        tol = np.full(len(E), ENERGY_TOL[ok.FP64_FIELDS])
    else:
        # FP32 spectra: the self part carries the transform's ~1e-7 relative error
        assert np.abs(D - Do).max() <= 5e-7 * np.abs(Do).max() + 1e-6
        tol = np.full(len(E), ENERGY_TOL[ok.FP32_FIELDS])
    assert np.all(np.abs(E - Eo) <= tol), (np.abs(E - Eo), tol)
    assert np.all(np.abs(Ec - Eco).max(axis=1) <= tol), (np.abs(Ec - Eco).max(axis=1), tol)
    # the approximation differs from the exact energy of an extended defect
    assert np.abs(E - Ex).max() > 1e-4


def test_dipole_tables_leave_the_trajectory_unchanged():
    """Computing dipole energies between steps (which builds their tables once) does not
    change the kinetics: same positions and statistics as a grid that never does."""
    w = config_small()
    a, b = make_grid(w), make_grid(w)
    a.step(w.T_K, 4)
    a.dipole_energies()
    sa = a.step(w.T_K, 4)
    b.step(w.T_K, 4)
    sb = b.step(w.T_K, 4)
    assert np.array_equal(a.get_positions(), b.get_positions())
    assert sa['events'] == sb['events'] and sa['clock'] == sb['clock']
    assert np.array_equal(a.interaction_energies(), b.interaction_energies())
    a.close()
    b.close()


# ------------------------------------------------------------------ kinetics
def test_incremental_field_equals_fresh_voxelisation():
    w = config_small()
    g = make_grid(w)
    g.step(w.T_K, 25)
    g.step(w.T_K, 5, mode=ok.FIXED_DT)
    cur = g.get_defects()
    eps_inc = g.eigenstrain()
    g2 = make_grid(w)
    g2.set_defects(cur)
    eps_new = g2.eigenstrain()
    assert np.array_equal(eps_inc, eps_new)
    g.close()
    g2.close()


def test_long_run_at_full_size_stays_exact():
    """10 000 residence-time steps and 200 fixed-time steps (Algorithm 1) of the 256^3
    workload with 2000 defects: the eigenstrain updated move by move equals a fresh
    voxelisation of the final positions bit for bit, and so do the stress and every
    site and candidate energy (the solve of a field that was built incrementally and
    of a fresh one differ in nothing)."""
    w = config_large()
    g = make_grid(w)
    st = g.step(w.T_K, 10000)
    assert st['events'] == 10000
    st = g.step(w.T_K, 200, mode=ok.FIXED_DT)
    assert st['steps'] == 10200 and st['events'] > 10000
    fresh = make_grid(w)
    fresh.set_defects(g.get_defects())
    assert np.array_equal(g.eigenstrain(), fresh.eigenstrain())
    assert np.array_equal(g.solve_stress(), fresh.solve_stress())
    assert np.array_equal(g.interaction_energies(), fresh.interaction_energies())
    assert np.array_equal(g.candidate_energies()[0], fresh.candidate_energies()[0])
    g.close()
    fresh.close()


def test_residence_steps_follow_oracle_decisions():
    w = config_small()
    seed = 4242
    g = make_grid(w, seed=seed)
    defs = w.defects.copy()
    clock = 0.0
    for step in range(20):
        E = g.interaction_energies()
        Ec, _ = g.candidate_energies()
        before = g.get_defects()
        assert np.array_equal(before['pos'], defs['pos'])
        i, j, dt, R = O.residence_step(defs, E, Ec, w.T_K, seed, step, w.n)
        st = g.step(w.T_K, 1)
        after = g.get_defects()
        assert np.array_equal(after['pos'], defs['pos']), step
        clock += dt
        assert abs(st['clock'] - clock) <= 1e-12 * clock
    assert g.stats()['events'] == 20
    g.close()


def test_fixed_dt_steps_follow_oracle_decisions():
    w = config_small()
    seed = 99
    g = make_grid(w, seed=seed)
    defs = w.defects.copy()
    dt = O.fixed_dt(defs, w.T_K)
    nev = 0
    for step in range(10):
        E = g.interaction_energies()
        Ec, _ = g.candidate_energies()
        mv = O.fixed_dt_step(defs, E, Ec, w.T_K, seed, step, w.n, dt)
        nev += len(mv)
        st = g.step(w.T_K, 1, mode=ok.FIXED_DT)
        assert np.array_equal(g.get_defects()['pos'], defs['pos']), step
        assert st['events'] == nev
        assert abs(st['dt_last'] - dt) <= 1e-12 * dt
    g.close()


def test_positions_roundtrip_and_update():
    w = config_small()
    g = make_grid(w)
    p = g.get_positions()
    assert np.array_equal(p, w.defects['pos'])
    p2 = p.copy()
    p2[3] = (p2[3] + 2) % 64
    g.set_positions(p2)
    assert np.array_equal(g.get_positions(), p2)
    moved = w.defects.copy()
    moved['pos'] = p2
    ref = zyx(O.eigenstrain_field(moved, w.n, w.voxel_nm))
    assert np.abs(g.eigenstrain() - ref).max() < 2e-7
    g.close()


def test_invalid_inputs_rejected():
    w = config_small()
    g = make_grid(w)
    bad = w.defects.copy()
    bad['pos'][0] = (1, 2, 3)               # mixed parity: not a bcc site
    with pytest.raises(ok.OkmcError) as e:
        g.set_defects(bad)
    assert e.value.code == ok.OKMC_EINVAL
    bad = w.defects.copy()
    bad['radius_nm'][0] = 10.0              # loop wider than half the box
    with pytest.raises(ok.OkmcError):
        g.set_defects(bad)
    bad = make_defects([1], np.array([[0, 0, 0]]), [0], [1.0], [0], [1.0], [ok.ONE_D])
    with pytest.raises(ok.OkmcError):       # <100> loops are immobile
        g.set_defects(bad)
    g.close()
    with pytest.raises(ok.OkmcError) as e:
        ok.Grid((64, 64, 64), 0.2855, *FE_CUBIC, hbm_budget=1 << 20)
    assert e.value.code == ok.OKMC_ENOMEM


@pytest.mark.parametrize('precision', [ok.FP32_FIELDS, ok.FP64_FIELDS])
def test_empty_defect_set(precision):
    """No defects (a degenerate input): the stress is zero everywhere, the energies are
    empty, a step is refused with OKMC_ESTATE, and defects set afterwards give the stress,
    energies and trajectory of a fresh grid bit for bit."""
    w = scaled_population((64, 64, 64), 8, seed=11, r111=(0.4, 1.0), r100=(0.4, 1.0))
    g = ok.Grid(w.n, w.voxel_nm, *w.C, precision=precision, seed=11)
    g.set_defects(w.defects[:0])
    assert not g.solve_stress().any()
    assert g.interaction_energies().shape == (0,)
    with pytest.raises(ok.OkmcError) as e:
        g.step(500.0, 1)
    assert e.value.code == ok.OKMC_ESTATE
    g.set_defects(w.defects)
    ref = make_grid(w, precision)
    assert np.array_equal(g.solve_stress(), ref.solve_stress())
    assert np.array_equal(g.candidate_energies()[0], ref.candidate_energies()[0])
    st, st_ref = g.step(500.0, 4), ref.step(500.0, 4)
    assert np.array_equal(g.get_positions(), ref.get_positions())
    assert st['clock'] == st_ref['clock']
    # only immobile defects (<100> loops): energies as usual, a step is refused
    still = make_defects([ok.LOOP_100, ok.LOOP_100], np.array([[10, 10, 10], [70, 40, 90]]), [0, 2], [0.8, 1.1], [0, 0],
                         [0.1, 0.1], [ok.IMMOBILE, ok.IMMOBILE])
    g.set_defects(still)
    assert np.all(np.isfinite(g.interaction_energies()))
    with pytest.raises(ok.OkmcError) as e:
        g.step(500.0, 1)
    assert e.value.code == ok.OKMC_ESTATE
    g.close()
    ref.close()


# ------------------------------------------------------------------ full-size configurations
def _sample(w, big_nm, n_other, seed):
    """Every loop with R > big_nm, the largest loops of each type up to 32 in all when
    fewer are that large, and n_other further defects drawn at random."""
    d = w.defects
    R = np.where(d['type'] != O.SIA_CLUSTER, d['radius_nm'], 0.0)
    big = [int(i) for i in np.argsort(-R) if R[i] > big_nm]
    if len(big) < 32:
        big = [int(i) for i in np.argsort(-R)[:32]]
    rest = np.setdiff1d(np.arange(len(d)), big)
    other = np.random.default_rng(seed).choice(rest, n_other, replace=False)
    return big + [int(i) for i in other]


def _full_size_oracle(w, big_nm, n_other, seed):
    from oracle_pool import sampled_energies
    C = O.stiffness_cubic(*w.C)
    ref = O.solve_stress(O.eigenstrain_field(w.defects, w.n, w.voxel_nm), C, w.voxel_nm)
    sample = _sample(w, big_nm, n_other, seed)
    return ref, sampled_energies(w.defects, sample, ref, w.n, w.voxel_nm, w.C)


def _check_sampled(w, picks, precision):
    g = make_grid(w, precision)
    sig = g.solve_stress()
    E = g.interaction_energies().copy()
    Ec, _ = g.candidate_energies()
    g.close()
    tol = ENERGY_TOL[precision]
    err = max(max(abs(E[i] - e0), np.abs(Ec[i] - ej).max()) for i, (e0, ej) in picks.items())
    assert err <= tol, (precision, err)
    return sig, E, Ec.copy()


@pytest.fixture(scope='module')
def medium_oracle():
    w = config_medium()
    return (w,) + _full_size_oracle(w, 3.5, 32, 3)


@pytest.mark.parametrize('precision', [ok.FP32_FIELDS, ok.FP64_FIELDS])
def test_medium_128_stress_and_sampled_energies(medium_oracle, precision):
    """The 128^3 workload: the whole stress field against the oracle, and the site and
    eight candidate energies of 64 defects (the 32 largest loops, 32 drawn at random)
    against the oracle's sigma - W route, at the flat bar (1e-4 eV FP32, 1e-8 FP64)."""
    w, ref, picks = medium_oracle
    assert len(picks) >= 64
    sig, _, _ = _check_sampled(w, picks, precision)
    assert rel_l2(sig, zyx(ref)) <= STRESS_TOL[precision]


@pytest.mark.parametrize('n,R', [(64, 2.5), (128, 4.0), (256, 4.0)])
def test_lone_defect_has_zero_interaction_energy(n, R):
    """A defect alone in the box interacts with nothing: E and every candidate energy
    are exactly 0, so what the FP32 path returns is its whole error (self term included)."""
    d = make_defects([0, 2], np.array([[n, n, n], [n + 1, n + 1, n + 1]]), [1, 0], [R, 0.0], [0, 4],
                     [0.1, 0.3], [ok.ONE_D, ok.THREE_D])
    for k in range(2):
        g = ok.Grid((n, n, n), 0.2855, *FE_CUBIC)
        g.set_defects(d[k:k + 1])
        E = g.interaction_energies()
        Ec, _ = g.candidate_energies()
        assert abs(E[0]) <= 1e-4 and np.abs(Ec).max() <= 1e-4, (n, R, k, E, np.abs(Ec).max())
        g.close()


@pytest.fixture(scope='module')
def large_oracle():
    w = config_large()
    return (w,) + _full_size_oracle(w, 3.5, 32, 4)


@pytest.mark.parametrize('precision', [ok.FP32_FIELDS, ok.FP64_FIELDS])
def test_large_256_stress_and_sampled_energies(large_oracle, precision):
    """The 256^3 workload in the configuration the benchmark times: the whole stress
    field against the oracle, and the site and eight candidate energies of every loop
    with R > 3.5 nm (115) and 32 defects drawn at random, against the oracle's sigma - W
    route, at the flat bar (1e-4 eV FP32, 1e-8 FP64)."""
    w, ref, picks = large_oracle
    assert len(picks) >= 64
    sig, _, _ = _check_sampled(w, picks, precision)
    assert rel_l2(sig, zyx(ref)) <= STRESS_TOL[precision]


def test_large_256_fp32_energies_of_every_defect_match_fp64_fields():
    """All 2000 site energies and 16000 candidate energies of the 256^3 workload: FP32
    fields against the FP64-field path (itself held to 1e-8 eV of the oracle above)."""
    w = config_large()
    out = {}
    for p in (ok.FP32_FIELDS, ok.FP64_FIELDS):
        g = make_grid(w, p)
        E = g.interaction_energies().copy()
        Ec, _ = g.candidate_energies()
        out[p] = (E, Ec.copy())
        g.close()
    dE = np.abs(out[ok.FP32_FIELDS][0] - out[ok.FP64_FIELDS][0]).max()
    dEc = np.abs(out[ok.FP32_FIELDS][1] - out[ok.FP64_FIELDS][1]).max()
    assert dE <= 1e-4 and dEc <= 1e-4, (dE, dEc)


# ------------------------------------------------------------------ incremental plane transforms
@pytest.mark.parametrize('mode', [ok.RESIDENCE, ok.FIXED_DT])
def test_incremental_plane_transforms_equal_fresh_solve(mode):
    """After steps that move defects, only the z-planes whose eigenstrain changed are
    transformed again; the stress equals, bit for bit, a fresh solve of the same
    configuration on a new grid (the fixed-point eigenstrain is exact, so every clean
    plane's input is the same)."""
    w = scaled_population((64, 64, 64), 40, seed=9, r111=(0.4, 1.2), r100=(0.4, 1.2))
    a = make_grid(w, seed=3)
    assert a.launch_shape()[0] == -1
    a.step(w.T_K, 25, mode=mode)
    moved = a.get_defects()
    assert not np.array_equal(moved['pos'], w.defects['pos'])
    sa = a.solve_stress()
    b = ok.Grid(w.n, w.voxel_nm, *w.C)
    b.set_defects(moved)
    sb = b.solve_stress()
    assert np.array_equal(sa, sb)
    assert np.array_equal(a.interaction_energies(), b.interaction_energies())
    a.close()
    b.close()


# ------------------------------------------------------------------ launch variants
@pytest.mark.parametrize('n', [(48, 48, 48), (96, 96, 64), (128, 128, 32), (160, 160, 32), (192, 192, 32),
                               (256, 256, 32), (320, 320, 32), (64, 64, 256), (48, 48, 320)])
def test_pass_variants_bitwise_equal(n):
    """Every launch variant of the FFT passes gives the same stress, bit for bit."""
    w = scaled_population(n, 20, seed=n[0], r111=(0.4, 1.0), r100=(0.4, 1.0))
    g = make_grid(w)
    cur, avail = g.variants()
    assert all((avail[p] >> cur[p]) & 1 for p in range(3))
    ref = None
    for p in range(3):
        for v in range(31):
            if not (avail[p] >> v) & 1:
                continue
            g.set_variant(p, v)
            if p == 0:
                g.set_defects(w.defects)  # every plane dirty, so the forward pass runs in full
            s = g.solve_stress()
            if ref is None:
                ref = s
            assert np.array_equal(s, ref), (p, v)
        g.set_variant(p, cur[p])
    with pytest.raises(ok.OkmcError):
        g.set_variant(2, 30)
    g.close()


def test_bulk_copy_wait_gives_up_with_a_status(monkeypatch):
    """The TMA-staged pencil pass waits on its copies with a bounded wait.  A test hook
    makes it expect 16 bytes more than its copies bring, so the wait runs out: every CTA
    records error code 6 and returns, the call that synchronises reports OKMC_ETIMEOUT,
    and the context stays usable (a fresh grid solves to the same stress as variant 0)."""
    w = scaled_population((32, 32, 32), 6, seed=5, r111=(0.4, 1.0), r100=(0.4, 1.0))
    monkeypatch.setenv('OKMC_VARIANTS', '0,0,0')
    monkeypatch.setenv('OKMC_TMA_EXTRA_TX', '16')
    g = make_grid(w)  # self terms by variant 0
    if not (g.variants()[1][1] >> 2) & 1:
        g.close()
        pytest.skip('no tensor maps on this device')
    g.set_variant(1, 2)
    t0 = time.time()
    with pytest.raises(ok.OkmcError) as ei:
        g.solve_stress()
    assert ei.value.code == ok.OKMC_ETIMEOUT, ei.value
    assert 0.4 < time.time() - t0 < 30.0
    g.close()
    monkeypatch.delenv('OKMC_TMA_EXTRA_TX')
    g = make_grid(w)
    ref = g.solve_stress()
    g.set_variant(1, 2)
    g.set_defects(w.defects)
    assert np.array_equal(g.solve_stress(), ref)
    g.close()


def test_variants_pinned_by_environment(monkeypatch):
    """OKMC_VARIANTS=a,b,c pins each pass's variant where it exists (no timing), and
    steps captured on a pinned grid follow the tuned grid's trajectory bit for bit."""
    w = scaled_population((64, 64, 64), 8, seed=3, r111=(0.4, 1.0), r100=(0.4, 1.0))
    ref = make_grid(w)
    st_ref = ref.step(500.0, 3)
    monkeypatch.setenv('OKMC_VARIANTS', '1,1,4')
    g = make_grid(w)
    cur, avail = g.variants()
    assert cur == [v if (avail[p] >> v) & 1 else 0 for p, v in enumerate((1, 1, 4))]
    st = g.step(500.0, 3)
    assert np.array_equal(g.get_positions(), ref.get_positions())
    assert st['events'] == st_ref['events'] and st['clock'] == st_ref['clock']
    assert np.array_equal(g.interaction_energies(), ref.interaction_energies())
    g.close()
    ref.close()
    monkeypatch.setenv('OKMC_VARIANTS', '0,0,30')  # variant 30 exists for no pass
    g = make_grid(w)
    assert g.variants()[0] == [0, 0, 0]
    g.close()


_TUNE_SCRIPT = r"""
import json, sys
sys.path.insert(0, sys.argv[1])
from paper_2403_09158_gb300 import okmc as ok
ok.load()
g = ok.Grid((sys.argv[2] and int(sys.argv[2]) or 96,) * 3, 0.2855, 243.0, 145.0, 116.0)
print(json.dumps(g.variants()))
g.close()
"""


def _tune_run(tmp_path, cache, edge=96):
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, OKMC_TUNE_CACHE=str(cache))
    env.pop('OKMC_VARIANTS', None)
    env.pop('OKMC_TUNE', None)
    r = subprocess.run([sys.executable, '-c', _TUNE_SCRIPT, root, str(edge)], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_tuner_picks_persist_across_processes(tmp_path):
    """The tuner writes its picks per device and grid shape to the JSON cache file; a new
    process with the same file adopts the recorded picks (a planted valid pick shows that
    the file, not a new timing, decided); an unreadable file counts as empty."""
    import json
    cache = tmp_path / 'sub' / 'tune.json'
    cur, avail = _tune_run(tmp_path, cache)
    data = json.loads(cache.read_text())
    keys = [k for k in data if '|96x96x96|' in k]
    assert len(keys) == 1 and data[keys[0]] == cur
    # plant another existing inverse-pass variant and check the next process takes it
    other = [v for v in range(31) if (avail[2] >> v) & 1 and v != cur[2]]
    assert other
    data[keys[0]] = [cur[0], cur[1], other[0]]
    cache.write_text(json.dumps(data))
    cur2, _ = _tune_run(tmp_path, cache)
    assert cur2 == [cur[0], cur[1], other[0]]
    cache.write_text('{ not json')
    cur3, _ = _tune_run(tmp_path, cache)
    assert all((avail[p] >> cur3[p]) & 1 for p in range(3))
    assert '|96x96x96|' in cache.read_text()


# ------------------------------------------------------------------ graphs and batches
def test_graph_replay_equals_kernel_by_kernel():
    w = config_small()
    a = make_grid(w, seed=5)
    b = make_grid(w, seed=5)
    b.set_graphs(False)
    for mode in (ok.RESIDENCE, ok.FIXED_DT):
        sa = a.step(w.T_K, 15, mode=mode)
        sb = b.step(w.T_K, 15, mode=mode)
        assert np.array_equal(a.get_positions(), b.get_positions())
        assert sa['clock'] == sb['clock'] and sa['events'] == sb['events']
    a.close()
    b.close()


def test_batch_replicas_equal_alone():
    """Replicas of uneven size (fast and generic passes) advanced by one graph per
    step give the same trajectory as each replica stepped alone."""
    small = dict(r111=(0.4, 1.0), r100=(0.4, 1.0))
    cases = [scaled_population((32, 32, 32), 12, seed=1, **small), scaled_population((64, 64, 64), 40, seed=2, **small),
             scaled_population((48, 32, 80), 20, seed=3, r111=(0.4, 1.0), r100=(0.4, 1.0))]
    Ts = [300.0, 450.0, 600.0]
    alone, mixed = [], []
    for w, T in zip(cases, Ts):
        g = ok.Grid(w.n, w.voxel_nm, *w.C, seed=77)
        g.set_defects(w.defects)
        st = g.step(T, 12)
        alone.append((g.get_positions(), st, g.interaction_energies()))
        g.close()
    grids = []
    for w in cases:
        g = ok.Grid(w.n, w.voxel_nm, *w.C, seed=77)
        g.set_defects(w.defects)
        grids.append(g)
    batch = ok.Batch(grids)
    batch.step(Ts, 5)
    stats = batch.step(Ts, 7)
    for (pos, st, E), g, s in zip(alone, grids, stats):
        assert np.array_equal(g.get_positions(), pos)
        assert s['clock'] == st['clock'] and s['events'] == st['events'] == 12
        assert np.array_equal(g.interaction_energies(), E)
    batch.close()
    for g in grids:
        g.close()


@pytest.mark.parametrize('mode', [ok.BATCH_KERNELS, ok.BATCH_GRAPHS])
def test_batched_kernels_equal_alone(mode):
    """An ensemble of replicas of uneven edges (64, 96, 128, 160, 192; one in fixed-time-step
    mode) advanced by the batched persistent kernels (one per stage and edge class over
    work lists) or by per-replica graph branches gives each replica its solo trajectory
    bit for bit."""
    small = dict(r111=(0.4, 1.2), r100=(0.4, 1.2))
    edges = [64, 96, 128, 64, 160, 192]
    cases = [scaled_population((e, e, e), 10 + 4 * k, seed=20 + k, **small) for k, e in enumerate(edges)]
    Ts = [300.0 + 50.0 * k for k in range(len(cases))]
    modes = [ok.RESIDENCE] * len(cases)
    modes[3] = ok.FIXED_DT
    alone = []
    for w, T, m in zip(cases, Ts, modes):
        g = ok.Grid(w.n, w.voxel_nm, *w.C, seed=91)
        g.set_defects(w.defects)
        st = g.step(T, 9, mode=m)
        Ec, _ = g.candidate_energies()
        alone.append((g.get_positions(), st, g.interaction_energies().copy(), Ec.copy()))
        g.close()
    grids = []
    for w in cases:
        g = ok.Grid(w.n, w.voxel_nm, *w.C, seed=91)
        g.set_defects(w.defects)
        grids.append(g)
    batch = ok.Batch(grids, mode=mode)
    batch.step(Ts, 4, mode=modes)
    assert batch.mode() == mode
    stats = batch.step(Ts, 5, mode=modes)
    for (pos, st, E, Ec), g, s in zip(alone, grids, stats):
        assert np.array_equal(g.get_positions(), pos)
        assert s['clock'] == st['clock'] and s['events'] == st['events'] and s['steps'] == st['steps']
        assert np.array_equal(g.interaction_energies(), E)
        assert np.array_equal(g.candidate_energies()[0], Ec)
    batch.close()
    for g in grids:
        g.close()


def test_batched_kernels_refuse_unsupported_edges():
    """BATCH_KERNELS with a replica outside the supported edges fails with EINVAL; AUTO
    falls back to graph branches."""
    w = scaled_population((48, 48, 48), 6, seed=5, r111=(0.4, 1.0), r100=(0.4, 1.0))
    g = ok.Grid(w.n, w.voxel_nm, *w.C, seed=3)
    g.set_defects(w.defects)
    b = ok.Batch([g], mode=ok.BATCH_KERNELS)
    with pytest.raises(ok.OkmcError) as e:
        b.step([400.0], 1)
    assert e.value.code == ok.OKMC_EINVAL
    b.close()
    b = ok.Batch([g])
    b.step([400.0], 1)
    assert b.mode() == ok.BATCH_GRAPHS
    b.close()
    g.close()


# ------------------------------------------------------------------ dislocation lines (field dislocation mechanics)
def _dislocation_case(n, h):
    """A clockwise 1/2[111] loop (off-grid centre, 48 vertices) and one period of a
    straight mixed dislocation along y, with their Burgers vectors."""
    n111 = np.ones(3) / np.sqrt(3.0)
    L = np.asarray(n) * h
    loop = O.circle_points(np.array([0.41, 0.37, 0.52]) * L, n111, 1.1, 48)[::-1]
    line = np.array([[0.2 * L[0], 0.3, 0.6 * L[2]], [0.2 * L[0], 0.3 + L[1], 0.6 * L[2]]])
    return [(loop, 0.5 * h * np.ones(3), True), (line, 0.5 * h * np.array([1.0, -1.0, 1.0]), False)]


def _oracle_dislocation_eigenstrain(lines, n, h, ds_max):
    """Nye tensor of every line (Eq. Nye2), Eq. eq_EIG_fourier with Eq. plastic_0 at xi = 0
    for the closed ones: A = -1/2 sum x_a x x_{a+1} for a line running clockwise about A."""
    alpha = sum(O.nye_tensor(p, b, n, h, closed=c, ds_max=ds_max) for p, b, c in lines)
    V = np.prod(n) * h ** 3
    U0 = np.zeros((3, 3))
    for p, b, c in lines:
        if c:
            A = -0.5 * np.sum(np.cross(p, np.roll(p, -1, axis=0)), axis=0)
            U0 += (np.outer(b, A) + np.outer(A, b)) / (2.0 * V)
    return O.dislocation_eigenstrain6(alpha, h, U0)


@pytest.mark.parametrize('precision,n', [(ok.FP64_FIELDS, (32, 48, 32)), (ok.FP32_FIELDS, (32, 48, 32)),
                                         (ok.FP32_FIELDS, (64, 64, 64))])
def test_dislocation_eigenstrain_stress_and_energies_match_oracle(precision, n):
    """Plastic strain of dislocation lines (Eqs. Nye2, eq_EIG_fourier, plastic_0), its
    stress, and the energies of defects in the lines' field, against the oracle."""
    h, ds_max = 0.2855, 0.27 * 0.2855   # ds_max keeps L / ds_max away from integers
    lines = _dislocation_case(n, h)
    eps_d = _oracle_dislocation_eigenstrain(lines, n, h, ds_max)
    C = O.stiffness_cubic(*FE_CUBIC)
    g = ok.Grid(n, h, *FE_CUBIC, precision=precision, seed=3)
    g.set_dislocations(lines, ds_max_nm=ds_max)
    eps = g.eigenstrain()
    ref = zyx(eps_d)
    if precision == ok.FP64_FIELDS:
        assert np.abs(eps - ref).max() <= 1e-9 * np.abs(ref).max()
    else:
        assert rel_l2(eps, ref) <= 1e-5 and np.abs(eps - ref).max() <= 1e-5 * np.abs(ref).max()
    sig_o = O.solve_stress(eps_d, C, h)
    assert rel_l2(g.solve_stress(), zyx(sig_o)) <= STRESS_TOL[precision]
    # two defects in the lines' field: E_i from sigma of (lines + the other defect)
    defs = make_defects([O.LOOP_111, O.SIA_CLUSTER], np.array([[24, 60, 16], [41, 21, 47]]), [1, 0], [0.6, 0.0],
                        [0, 3], [0.1, 0.3], [1, 2])
    g.set_defects(defs)
    E, Ec = g.interaction_energies(), g.candidate_energies()[0]
    for i in range(2):
        sig = O.solve_stress(O.eigenstrain_field(defs, n, h, exclude={i}) + eps_d, C, h)
        assert abs(E[i] - O.energy_of_stencil(defs[i], defs[i]['pos'], sig, h)) <= ENERGY_TOL[precision]
        eco = [O.energy_of_stencil(defs[i], Y, sig, h) for Y in O.candidate_positions(defs[i]['pos'])]
        assert np.abs(Ec[i] - eco).max() <= ENERGY_TOL[precision]
    g.close()


def test_dislocation_background_survives_steps_and_can_be_removed():
    """The lines' plastic strain stays under the incremental updates of a trajectory:
    after steps, the field equals a fresh grid's with the defects at their new sites,
    whichever of set_dislocations and set_defects came first; removing the lines leaves
    the defects' field alone."""
    n, h = (64, 64, 64), 0.2855
    lines = _dislocation_case(n, h)
    defs = make_defects([O.LOOP_111, O.SIA_CLUSTER, O.SIA_CLUSTER],
                        np.array([[40, 64, 90], [81, 41, 21], [20, 100, 60]]), [0, 1, 2], [0.8, 0.0, 0.0],
                        [0, 2, 1], [0.1, 0.3, 0.3], [1, 2, 2])
    a = ok.Grid(n, h, *FE_CUBIC, seed=5)
    a.set_dislocations(lines)
    a.set_defects(defs)
    a.step(300.0, 30)
    moved = defs.copy()
    moved['pos'] = a.get_positions()
    assert not np.array_equal(moved['pos'], defs['pos'])
    b = ok.Grid(n, h, *FE_CUBIC, seed=5)
    b.set_defects(moved)
    b.set_dislocations(lines)
    assert np.array_equal(a.eigenstrain(), b.eigenstrain())
    assert np.array_equal(a.interaction_energies(), b.interaction_energies())
    a.set_dislocations([])
    c = ok.Grid(n, h, *FE_CUBIC, seed=5)
    c.set_defects(moved)
    assert np.array_equal(a.eigenstrain(), c.eigenstrain())
    for x in (a, b, c):
        x.close()
