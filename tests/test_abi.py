"""The C ABI library builds, loads and exports every symbol include/okmc.h declares;
ctypes structures match the C structure layouts.  No GPU compute is called."""
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

import __graft_entry__
from paper_2403_09158_gb300 import okmc as ok
from paper_2403_09158_gb300.workload import DEFECT_DTYPE

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, 'include', 'okmc.h')


def declared():
    txt = open(HEADER).read()
    txt = re.sub(r'/\*.*?\*/', '', txt, flags=re.S)
    return sorted(set(re.findall(r'\b(okmc_[a-z_]+)\s*\(', txt)))


@pytest.fixture(scope='module')
def lib():
    __graft_entry__.build()
    return ok.load()


def test_exports_every_declared_symbol(lib):
    names = declared()
    assert len(names) >= 20
    out = subprocess.run(['nm', '-D', '--defined-only', ok.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r' T (okmc_\w+)', out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    assert sorted(ok.EXPORTED) == names
    for n in names:
        assert hasattr(lib, n)


def test_struct_layouts_match_c():
    src = r'''
#include <stdio.h>
#include <stddef.h>
#include "okmc.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(okmc_grid_desc), sizeof(okmc_defect), sizeof(okmc_step_params),
         sizeof(okmc_step_stats), offsetof(okmc_grid_desc, voxel_nm), offsetof(okmc_grid_desc, stream),
         offsetof(okmc_defect, radius_nm));
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(okmc_server_desc), sizeof(okmc_request), sizeof(okmc_result),
         sizeof(okmc_server_stats), offsetof(okmc_request, params), offsetof(okmc_request, positions),
         offsetof(okmc_result, stats));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, 'l.c')
        open(c, 'w').write(src)
        exe = os.path.join(d, 'l')
        subprocess.run(['gcc', '-I', os.path.join(ROOT, 'include'), c, '-o', exe], check=True)
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    import ctypes as C
    assert vals[0] == C.sizeof(ok.GridDesc)
    assert vals[1] == DEFECT_DTYPE.itemsize == 48
    assert vals[2] == C.sizeof(ok.StepParams)
    assert vals[3] == C.sizeof(ok.StepStats)
    assert vals[4] == ok.GridDesc.voxel_nm.offset
    assert vals[5] == ok.GridDesc.stream.offset
    assert vals[6] == DEFECT_DTYPE.fields['radius_nm'][1]
    assert vals[7] == C.sizeof(ok.ServerDesc)
    assert vals[8] == C.sizeof(ok.Request)
    assert vals[9] == C.sizeof(ok.Result)
    assert vals[10] == C.sizeof(ok.ServerStats)
    assert vals[11] == ok.Request.params.offset
    assert vals[12] == ok.Request.positions.offset
    assert vals[13] == ok.Result.stats.offset


def test_null_handle_errors_without_gpu(lib):
    # argument checks run on the host before any CUDA call
    assert lib.okmc_grid_destroy(None) == ok.OKMC_OK
    assert lib.okmc_last_error(None) == b'null handle'
    assert lib.okmc_solve_stress(None, None, 0) == ok.OKMC_EINVAL
    assert lib.okmc_set_dislocations(None, None, None, None, None, 0, 0.0) == ok.OKMC_EINVAL
    d = ok.GridDesc()
    d.n[:] = (20, 32, 32)       # 20 is not a multiple of 16
    d.voxel_nm, d.C11, d.C12, d.C44 = 0.2855, 243.0, 145.0, 116.0
    import ctypes as C
    h = C.c_void_p()
    assert lib.okmc_grid_create(C.byref(d), C.byref(h)) == ok.OKMC_EINVAL
    d.n[:] = (32, 32, 32)
    d.C44 = -1.0
    assert lib.okmc_grid_create(C.byref(d), C.byref(h)) == ok.OKMC_EINVAL
    d.C44, d.k0_mode = 116.0, 7
    assert lib.okmc_grid_create(C.byref(d), C.byref(h)) == ok.OKMC_EINVAL


def test_server_and_estimate_argument_checks_without_gpu(lib):
    import ctypes as C
    assert lib.okmc_server_destroy(None) == ok.OKMC_OK
    assert lib.okmc_server_last_error(None) == b'null server'
    assert lib.okmc_server_create(None, None) == ok.OKMC_EINVAL
    d = ok.ServerDesc(0, 0, 0)  # no lanes
    h = C.c_void_p()
    assert lib.okmc_server_create(C.byref(d), C.byref(h)) == ok.OKMC_EINVAL
    assert lib.okmc_server_submit(None, None, None) == ok.OKMC_EINVAL
    assert lib.okmc_server_wait(None, 1, 0, None) == ok.OKMC_EINVAL
    assert lib.okmc_set_kinetic_state(None, None) == ok.OKMC_EINVAL
    # field bytes of a 256^3 FP32 grid on the register-FFT path: int32 eigenstrain,
    # FP32 stress, two half spectra, plus small tables
    n = 256
    b = ok.estimate_field_bytes((n, n, n), 0.2855, 243.0, 145.0, 116.0)
    fields = 6 * n ** 3 * 4 * 2 + 2 * 6 * n * (n // 2 + 1) * n * 8
    assert fields <= b <= fields + (1 << 20)
    bd = ok.estimate_field_bytes((n, n, n), 0.2855, 243.0, 145.0, 116.0, precision=ok.FP64_FIELDS)
    assert 6 * n ** 3 * 8 * 2 + 6 * n * (n // 2 + 1) * n * 16 <= bd
    assert ok.estimate_field_bytes((0, 8, 8), 0.2855, 243.0, 145.0, 116.0) == 0


def test_product_path_does_not_import_oracle():
    pkg = os.path.join(ROOT, 'paper_2403_09158_gb300')
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith(('.py', '.cu', '.cuh', '.h')):
                txt = open(os.path.join(dirpath, f)).read()
                assert 'import oracle' not in txt and 'from oracle' not in txt, f


def test_isotropic_stiffness_matches_the_lame_relations(lib):
    import oracle as O
    for mu, nu in ((82.0, 0.29), (100.0, 0.0), (50.0, -0.4), (30.0, 0.49)):
        got = ok.isotropic_stiffness(mu, nu)
        ref = O.isotropic_cubic_constants(mu, nu)
        assert np.allclose(got, ref, rtol=1e-15, atol=0)
        assert abs(got[2] - 0.5 * (got[0] - got[1])) <= 1e-12 * got[0]
    for mu, nu in ((0.0, 0.3), (-1.0, 0.3), (80.0, 0.5), (80.0, -1.0), (float('nan'), 0.3)):
        with pytest.raises(ok.OkmcError):
            ok.isotropic_stiffness(mu, nu)


def test_kinetics_workload_geometry():
    """The two-loop kinetics setting (Sec. 5.1): both loops on bcc sites (all three
    half-lattice coordinates of one parity), 1D glide along [111], separated by about
    10 nm along [1-10] and by x_rel along [111]."""
    from paper_2403_09158_gb300.workload import LOOP_111, ONE_D, config_kinetics
    for x_rel in (10.0, 20.0):
        w = config_kinetics(x_rel)
        d = w.defects
        assert list(d['type']) == [LOOP_111, LOOP_111] and list(d['mobility']) == [ONE_D, ONE_D]
        assert list(d['axis']) == [0, 0] and np.allclose(d['radius_nm'], 3.3) and np.allclose(d['Em_eV'], 0.1)
        for p in d['pos']:
            assert len({int(v) % 2 for v in p}) == 1
            assert np.all((p >= 0) & (p < 2 * np.asarray(w.n)))
        sep = (d['pos'][1] - d['pos'][0]) * 0.5 * w.voxel_nm
        along = sep @ np.ones(3) / np.sqrt(3.0)
        across = sep @ np.array([1.0, -1.0, 0.0]) / np.sqrt(2.0)
        assert abs(along - x_rel) < 0.25 and abs(across - 10.0) < 0.25
        assert abs(sep @ np.array([1.0, 1.0, -2.0])) < 1e-12       # no offset along [11-2]
        assert np.isclose(w.extra['x_rel_nm'], along) and np.isclose(w.extra['z_rel_nm'], across)


def test_dislocation_workload_geometry():
    """The loops-near-a-dislocation setting (Sec. 5.2): the edge line runs along y =
    [-1-12] through the box centre for one period (its end a lattice translate of its
    start) with b = (a0/2)[111] normal to it; the loops sit on bcc sites on both sides
    of the line (z = -/+ the same offset along [1-10], y = 0), x_rel apart along [111]
    with their centre of mass x_c from the line."""
    from paper_2403_09158_gb300.workload import config_dislocation_loops, frame_111
    X, Y, Z = frame_111()
    for x_c in (20.0, 30.0):
        w = config_dislocation_loops(x_c)
        (pts, b, closed), = w.extra['lines']
        n, h = np.asarray(w.n), w.voxel_nm
        assert not closed and pts.shape == (2, 3)
        per = (pts[1] - pts[0]) / h
        assert np.allclose(per, np.round(per)) and np.all(np.mod(np.round(per), n) == 0)
        assert np.allclose(np.cross(per, Y), 0.0) and abs(b @ per) < 1e-12
        assert np.allclose(b, 0.5 * h * np.ones(3))
        centre = 0.5 * n * h
        assert np.allclose(np.cross(centre - pts[0], per), 0.0)            # the line passes through the centre
        rel = [(p * 0.5 * h - centre) for p in w.defects['pos']]
        for p in w.defects['pos']:
            assert len({int(v) % 2 for v in p}) == 1
        zs = [r @ Z for r in rel]
        assert abs(zs[0] + zs[1]) < 1e-9 and abs(abs(zs[0]) - 5.0) < 0.2
        assert all(abs(r @ Y) < 1e-9 for r in rel)
        xs = [r @ X for r in rel]
        assert abs(0.5 * (xs[0] + xs[1]) - x_c) < 0.3 and abs(xs[1] - xs[0] - 10.0) < 0.3


def test_python_marshalling_of_dislocations_and_point_dipoles():
    """Grid.set_dislocations, point_dipole_energies and shift_energies hand the C calls flat,
    contiguous arrays in the documented layouts (checked with a stand-in library that
    reads the pointers during the call; no GPU)."""
    import ctypes as C
    seen = {}

    def rd(addr, ctype, count):
        return np.ctypeslib.as_array(C.cast(addr, C.POINTER(ctype)), shape=(count,)).copy()

    class FakeLib:
        def okmc_set_dislocations(self, h, pts, counts, closed, b, n, ds):
            cnt = rd(counts, C.c_int32, n)
            seen['counts'], seen['closed'] = cnt, rd(closed, C.c_int32, n)
            seen['pts'] = rd(pts, C.c_double, 3 * int(cnt.sum())).reshape(-1, 3)
            seen['b'], seen['ds'] = rd(b, C.c_double, 3 * n).reshape(-1, 3), ds
            return ok.OKMC_OK

        def okmc_point_dipole_energies(self, h, pos, P, m, E, on_device):
            seen['pos'], seen['P'] = rd(pos, C.c_int32, 3 * m).reshape(-1, 3), rd(P, C.c_double, 6 * m).reshape(-1, 6)
            out = np.ctypeslib.as_array(C.cast(E, C.POINTER(C.c_double)), shape=(m,))
            out[:] = np.arange(m) + 0.5
            seen['dev'] = on_device
            return ok.OKMC_OK

        def okmc_shift_energies(self, h, i, X, m, E, on_device):
            seen['i'], seen['X'] = i, rd(X, C.c_double, 3 * m).reshape(-1, 3)
            np.ctypeslib.as_array(C.cast(E, C.POINTER(C.c_double)), shape=(m,))[:] = -np.arange(m)
            return ok.OKMC_OK

    g = object.__new__(ok.Grid)
    g.lib, g.h = FakeLib(), C.c_void_p(1)
    loop = np.arange(12, dtype=np.float32).reshape(4, 3)           # converted to float64
    line = [[0.0, 0.0, 0.0], [0.0, 5.0, 0.0]]
    g.set_dislocations([(loop, (1, 2, 3), True), (line, np.array([0.5, 0.0, 0.5]), False)], ds_max_nm=0.05)
    assert list(seen['counts']) == [4, 2] and list(seen['closed']) == [1, 0]
    assert np.array_equal(seen['pts'], np.vstack([loop.astype(np.float64), line]))
    assert np.array_equal(seen['b'], [[1, 2, 3], [0.5, 0.0, 0.5]]) and seen['ds'] == 0.05
    pos = np.array([[2, 4, 6], [1, 3, 5]], dtype=np.int64)
    E = g.point_dipole_energies(pos, [1, 2, 3, 4, 5, 6])
    assert np.array_equal(seen['pos'], pos) and np.array_equal(seen['P'], [[1, 2, 3, 4, 5, 6]] * 2)
    assert np.array_equal(E, [0.5, 1.5]) and seen['dev'] == 0
    X = np.arange(9, dtype=np.float32).reshape(3, 3) * 0.1
    assert np.array_equal(g.shift_energies(2, X), [0.0, -1.0, -2.0])
    assert seen['i'] == 2 and np.array_equal(seen['X'], X.astype(np.float64))
    g.h = None
