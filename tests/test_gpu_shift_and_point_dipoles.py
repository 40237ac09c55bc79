"""Energies of probes of the field through the C ABI against the oracle: a defect moved
to continuous positions by the shift theorem (Sec. 3.3, Eq. shift; the Parseval sum of
the elastic-strain form with the defect's class-0 reference field moved by
exp(-i xi.X)), and point defects of given dipole tensor (Eq. interaction_energy4, Table 1).

Bars: 1e-8 eV with FP64 fields, 1e-4 eV with FP32 fields.
"""
import numpy as np
import pytest

import __graft_entry__
import oracle as O
from paper_2403_09158_gb300 import okmc as ok
from paper_2403_09158_gb300.workload import FE_CUBIC, make_defects

pytestmark = pytest.mark.gpu

TOL = {ok.FP32_FIELDS: 1e-4, ok.FP64_FIELDS: 1e-8}


@pytest.fixture(scope='module', autouse=True)
def _lib():
    __graft_entry__.build()
    ok.load()


@pytest.mark.parametrize('precision,k0', [(ok.FP64_FIELDS, ok.MEAN_STRESS_ZERO), (ok.FP32_FIELDS, ok.MEAN_STRESS_ZERO),
                                          (ok.FP64_FIELDS, ok.MEAN_STRAIN_ZERO)])
def test_shift_energies_match_oracle(precision, k0):
    """Three defects (a loop on a class-1 site, a loop and an SIA cluster on class-0
    sites) in a 32x48x32 box with a dislocation line; each defect moved to ten
    continuous positions (two passes of the position loop), against the oracle."""
    n, h = (32, 48, 32), 0.2855
    defs = make_defects([O.LOOP_111, O.LOOP_111, O.SIA_CLUSTER], np.array([[21, 41, 33], [40, 20, 12], [10, 70, 50]]),
                        [0, 2, 0], [0.8, 0.5, 0.0], [0, 0, 4], [0.1, 0.1, 0.3], [1, 1, 2])
    L = np.asarray(n) * h
    line = np.array([[0.55 * L[0], 0.1, 0.85 * L[2]], [0.55 * L[0], 0.1 + L[1], 0.85 * L[2]]])
    lines = [(line, 0.5 * h * np.ones(3), False)]
    C = O.stiffness_cubic(*FE_CUBIC)
    g = ok.Grid(n, h, *FE_CUBIC, k0_mode=k0, precision=precision, seed=9)
    g.set_dislocations(lines)
    g.set_defects(defs)
    eps_d = O.dislocation_eigenstrain6(O.nye_tensor(line, lines[0][1], n, h, closed=False), h)
    rng = np.random.default_rng(17)
    for i in range(3):
        X0 = defs['pos'][i] * h / 2.0
        X = X0[None, :] + rng.uniform(-0.6, 0.6, size=(10, 3))
        X[0] = X0
        E = g.shift_energies(i, X)
        ref = O.elastic_strain_spectrum(defs[i], n, h, C, k0)
        s_ext = O.solve_stress(O.eigenstrain_field(defs, n, h, exclude={i}) + eps_d, C, h, k0)
        Eo = np.array([O.energy_shift_theorem(ref, x, s_ext, h) for x in X])
        assert np.abs(E - Eo).max() <= TOL[precision], (i, np.abs(E - Eo))
        assert np.ptp(Eo) > 1e-3
    g.close()


def test_shift_energy_at_a_site_is_the_stencil_energy_on_the_grid():
    """A class-0 defect moved by whole voxels lands on its own stencil: the shift-theorem
    energy at its site equals the stencil energy (up to the Nyquist terms of the even
    edges, small here), and the call leaves the kinetics untouched."""
    n, h = (48, 48, 48), 0.2855
    defs = make_defects([O.LOOP_111, O.SIA_CLUSTER], np.array([[40, 50, 30], [60, 20, 70]]), [1, 0], [0.9, 0.0],
                        [0, 3], [0.1, 0.3], [1, 2])
    a, b = (ok.Grid(n, h, *FE_CUBIC, precision=ok.FP64_FIELDS, seed=4) for _ in range(2))
    for g in (a, b):
        g.set_defects(defs)
    E = a.interaction_energies()
    Es = np.array([a.shift_energies(i, defs['pos'][i][None, :] * h / 2.0)[0] for i in range(2)])
    assert np.allclose(Es, E, rtol=2e-3, atol=1e-6), (Es, E)
    a.step(300.0, 5)
    b.step(300.0, 5)
    assert np.array_equal(a.get_positions(), b.get_positions())
    for g in (a, b):
        g.close()


@pytest.mark.parametrize('precision', [ok.FP64_FIELDS, ok.FP32_FIELDS])
def test_point_dipole_energies_match_oracle(precision):
    """Point defects of given dipole tensor (Table 1's <110> dumbbell and an arbitrary
    one) probing the field of a dislocation line and two defects (eps = C^-1 : sigma at
    the site centre), against the oracle; a site off the lattice is rejected."""
    n, h = (32, 48, 32), 0.2855
    L = np.asarray(n) * h
    line = np.array([[0.55 * L[0], 0.1, 0.85 * L[2]], [0.55 * L[0], 0.1 + L[1], 0.85 * L[2]]])
    lines = [(line, 0.5 * h * np.ones(3), False)]
    defs = make_defects([O.LOOP_111, O.SIA_CLUSTER], np.array([[24, 60, 16], [41, 21, 47]]), [1, 0], [0.6, 0.0],
                        [0, 3], [0.1, 0.3], [1, 2])
    C = O.stiffness_cubic(*FE_CUBIC)
    g = ok.Grid(n, h, *FE_CUBIC, precision=precision, seed=3)
    g.set_dislocations(lines)
    g.set_defects(defs)
    eps_d = O.dislocation_eigenstrain6(O.nye_tensor(line, lines[0][1], n, h, closed=False), h)
    sig = O.solve_stress(O.eigenstrain_field(defs, n, h) + eps_d, C, h)
    pos = np.array([[10, 20, 30], [11, 21, 31], [0, 0, 0], [63, 95, 63], [30, 60, 20], [33, 7, 45]])
    P = np.stack([O.SIA_110_DIPOLE_EV] * 3 + [np.array([3.0, -1.0, 2.0, 0.5, -0.7, 1.1])] * 3)
    E = g.point_dipole_energies(pos, P)
    Eo = np.array([O.point_dipole_energy(P[k], pos[k], sig, C) for k in range(len(pos))])
    assert np.abs(E - Eo).max() <= TOL[precision], np.abs(E - Eo)
    assert np.abs(Eo).max() > 1e-3
    with pytest.raises(ok.OkmcError):
        g.point_dipole_energies(np.array([[10, 21, 30]]), P[:1])
    assert np.array_equal(g.point_dipole_energies(pos[:2], P[:2]), E[:2])
    g.close()
